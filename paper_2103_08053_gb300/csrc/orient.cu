// orient.cu -- rank-by-degree orientation and out-degree binning.
//
// Orientation (TRUST Sec. 2.2, rank-by-degree; Sec. 4.3 "after orientation"):
// an undirected edge {u,v} is kept once, as u -> v, iff
// (deg u, u) < (deg v, v) lexicographically, deg being the undirected
// degree. Every triangle then has exactly one vertex with both other vertices
// in its out-list, so Algorithm 1 run on N+ counts each triangle once.
//
// Kernels, in launch order (all HBM-streaming):
//   k_degree        deg[u] = row_ptr[u+1] - row_ptr[u]          (reads 8|4 B/row)
//   k_orient<count> kept[u] = #{v in N(u) : rank u < rank v}    (reads col + deg gather)
//   k_scan_*        dag_ptr = exclusive scan of kept (int64 carry, int32 out)
//   k_orient<compact> dag_col = kept neighbours, input order   (re-reads col, writes m)
// A warp owns 32 consecutive rows and walks their concatenated neighbour
// lists with coalesced 32-lane loads; each lane finds its row by a forward
// walk over the 33 row starts held in shared memory, and per-row positions
// come from ballots over the row segments of the 32 lanes (no atomics).
//
// Binning (Sec. 4.3 co-optimisation): d+ < 2 is skipped (no triangle can be
// closed), 2 <= d+ <= T_w goes to the warp-worker list, d+ > T_w becomes
// ceil(d+ / item_neighbors) thread-block work items (u, first neighbour).
#include "tc_internal.h"

namespace tcg {

namespace {

__device__ __forceinline__ unsigned lanemask_le(int lane) { return (2u << lane) - 1u; }
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// The graph owning global row `row`: the single graph, or for a batch the
// last graph whose vertex base is <= row (bases ascending, multiples of 32).
template <bool BATCH>
__device__ __forceinline__ GraphRef graph_of(int64_t row, const GraphRef& one, const GraphRef* __restrict__ gs,
                                             int k) {
    if (!BATCH) return one;
    int lo = 0, hi = k;  // first graph with vbase > row
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (gs[mid].vbase <= row) lo = mid + 1;
        else hi = mid;
    }
    return gs[lo - 1];
}

template <typename Off, bool BATCH>
__global__ void k_degree(GraphRef one, const GraphRef* __restrict__ gs, int k, int64_t total,
                         int32_t* __restrict__ deg, int32_t* __restrict__ hubs, int2* __restrict__ bnd,
                         long long entries, DevCounters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += stride) {
        const GraphRef G = graph_of<BATCH>(u, one, gs, k);
        const int64_t ul = u - G.vbase;
        long long d = 0;
        if (ul < G.n) {
            const Off* rp = static_cast<const Off*>(G.row_ptr);
            const long long a = (long long)rp[ul], b = (long long)rp[ul + 1];
            d = b - a;
            if (a < 0 || d < 0 || b > G.nnz || d > 0x7fffffffLL) {
                atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
                d = 0;
            }
        }
        deg[u] = (int32_t)d;
        if (bnd && u == total - 1)  // row-local DAG: the entries readable past the last list
            bnd[total] = make_int2((int32_t)entries, 0);
        if (d > HUB_DEGREE) hubs[atomicAdd(&ctr->n_hub, 1)] = (int32_t)u;
        else if (d > MID_DEGREE) hubs[total - 1 - atomicAdd(&ctr->n_mid, 1)] = (int32_t)u;  // from the back
    }
}

// L2 eviction hints (PTX createpolicy + ld.global.nc.L2::cache_hint). The
// orientation passes stream the neighbour lists once and gather a neighbour's
// degree for every entry: the lists are read evict-first and the degree
// gathers evict-last, so the streamed lists do not push the (much smaller)
// degree array out of L2.
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ldg_hint(const int32_t* a, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

constexpr int ORIENT_THREADS = 256;
constexpr int ORIENT_WARPS = ORIENT_THREADS / 32;
constexpr int ORIENT_UNROLL = 4;

// Virtual-combination owner map (as in the counting kernels, Sec. 4.2):
// lists held one per lane (inclusive prefix P, exclusive Pex, `listlane`
// marks lanes holding a non-empty list, compacted to the low lanes); for the
// window of combined indices [b, b+32), the list owning index b + lane.
__device__ __forceinline__ int owner_of(int b, int P, int Pex, bool listlane, unsigned le) {
    const int j0 = __popc(__ballot_sync(FULL, listlane && P <= b));
    const unsigned bit = listlane ? __funnelshift_lc(0u, 1u, (unsigned)(Pex - b)) : 0u;
    const unsigned starts = __reduce_or_sync(FULL, bit);
    return j0 + __popc(starts & le) - (int)(starts & 1u);
}

// COMPACT == false: kept[u] = out-degree (and the keep bits). COMPACT == true:
// write dag_col. Global row space [0, total); a batch pads every graph to a
// multiple of 32 rows, so a 32-row warp group never spans two graphs. deg,
// kept, dag_ptr and the DAG's neighbour ids are global (vbase + local id).
//
// A warp owns 32 consecutive rows. Its non-empty rows shorter than the hub
// threshold are compacted to the low lanes (row id, start, length), and their
// neighbour lists are walked as one virtually combined list, 32 entries per
// window, coalesced; a lane finds the row of its entry with owner_of. The row
// held by lane i counts its kept entries of a window with one popcount over
// the window's ballot restricted to its lanes; in the compaction pass, a kept
// entry's position is its row's next position (fetched from the row's lane)
// plus the kept entries before it in the row's part of the window.
template <typename Off, bool COMPACT, bool BATCH>
__global__ void __launch_bounds__(ORIENT_THREADS)
    k_orient(GraphRef one, const GraphRef* __restrict__ gs, int k, int64_t total, const int32_t* __restrict__ deg,
             int32_t* __restrict__ kept, const int32_t* __restrict__ dag_ptr, int32_t* __restrict__ dag_col,
             int64_t dag_cap, unsigned* __restrict__ kbits, int32_t* __restrict__ rdag, int2* __restrict__ bnd,
             int64_t g_lo, int64_t g_hi, DevCounters* ctr) {
    __shared__ long long s_a[ORIENT_WARPS][32];
    __shared__ int s_len[ORIENT_WARPS][32];
    __shared__ int s_rid[ORIENT_WARPS][32];
    if (COMPACT && ctr->err) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned le = lanemask_le(lane), lt = lanemask_lt(lane);
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // groups [g_lo, g_hi) of 32 rows (all of them, or one piece of a graph whose
    // neighbour lists arrive in pieces)
    for (int64_t g = g_lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < g_hi && g * 32 < total;
         g += nw) {
        const GraphRef G = graph_of<BATCH>(g * 32, one, gs, k);
        const Off* row_ptr = static_cast<const Off*>(G.row_ptr);
        const int32_t* col = G.col;
        const int64_t n = G.n, nnz = G.nnz, vb = G.vbase;
        const int64_t u0 = g * 32 - vb;  // local id of the group's first row
        const int nr = (int)(n - u0 < 32 ? (n - u0 > 0 ? n - u0 : 0) : 32);
        const int64_t row0 = BATCH ? g * 32 : u0;  // index of the group's first row in kept / dag_ptr
        if (nr == 0) {  // padding rows of a batch
            if (!COMPACT) {
                if (bnd) bnd[g * 32 + lane] = make_int2(0, 0);
                else kept[g * 32 + lane] = 0;
            }
            continue;
        }
        long long e = 0;
        if (lane == 0) e = (long long)row_ptr[u0 + nr];
        e = __shfl_sync(FULL, e, 0);
        const long long a = (lane < nr) ? (long long)row_ptr[u0 + lane] : e;
        long long nx = __shfl_down_sync(FULL, a, 1);
        if (lane == 31) nx = e;
        const bool bad = (lane < nr) && (a < 0 || nx < a || nx > nnz);
        if (__any_sync(FULL, bad)) {
            if (lane == 0) atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
            continue;
        }
        const long long len = nx - a;
        // rows walked here: non-empty and not hubs (the hub kernel takes those)
        const bool walk = lane < nr && len > 0 && len <= MID_DEGREE;
        if (!COMPACT && (BATCH || lane < nr) && !walk) {  // mid and hub rows: rewritten later
            if (bnd) bnd[row0 + lane] = make_int2((int)(G.ebase + a), 0);
            else kept[row0 + lane] = 0;
        }
        const unsigned wm = __ballot_sync(FULL, walk);
        if (wm == 0) continue;
        const bool hubless = __ballot_sync(FULL, lane < nr && len > MID_DEGREE) == 0;
        const int c = __popc(wm);
        if (walk) {
            const int p = __popc(wm & lt);
            s_a[w][p] = a;
            s_len[w][p] = (int)len;
            s_rid[w][p] = lane;
        }
        __syncwarp();
        const bool lst = lane < c;
        const long long ca = lst ? s_a[w][lane] : 0;
        const int cl = lst ? s_len[w][lane] : 0;
        const int rid = lst ? s_rid[w][lane] : 0;
        __syncwarp();
        int P = cl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, P, o);
            if (lane >= o) P += t;
        }
        const int tot = __shfl_sync(FULL, P, 31);
        const int Pex = P - cl;
        const long long bias = ca - Pex;  // col index of combined entry f of this row: bias + f
        const uint64_t pol_stream = l2_policy_first(), pol_keep = l2_policy_last();
        int cnt = (COMPACT && lst) ? dag_ptr[row0 + rid] : 0;  // compaction: the row's next output position
        for (int b0 = 0; b0 < tot; b0 += 32 * ORIENT_UNROLL) {
            // every load of the step first: ORIENT_UNROLL col reads, then their
            // degree gathers, so each lane has that many requests in flight
            int vq[ORIENT_UNROLL], dq[ORIENT_UNROLL], oq[ORIENT_UNROLL];
            long long atq[ORIENT_UNROLL];
#pragma unroll
            for (int q = 0; q < ORIENT_UNROLL; ++q) {
                const int bw = b0 + 32 * q;
                const int o = owner_of(bw, P, Pex, lst, le) & 31;
                oq[q] = o;
                const int f = bw + lane;
                atq[q] = __shfl_sync(FULL, bias, o) + f;
                vq[q] = (f < tot) ? ldg_hint(col + atq[q], pol_stream) : -1;
            }
            // the compaction pass reads the count pass's keep bits instead of
            // gathering the neighbours' degrees again
            const bool gather = !(COMPACT && kbits);
#pragma unroll
            for (int q = 0; q < ORIENT_UNROLL; ++q)
                dq[q] = (gather && (unsigned)vq[q] < (unsigned long long)n) ? ldg_hint(deg + vb + vq[q], pol_keep) : 0;
#pragma unroll
            for (int q = 0; q < ORIENT_UNROLL; ++q) {
                const int bw = b0 + 32 * q;
                if (bw >= tot) break;
                const int f = bw + lane;
                const bool act = f < tot;
                const int o = oq[q];
                const int du = __shfl_sync(FULL, cl, o);
                const int ur = __shfl_sync(FULL, rid, o);
                const int v = vq[q];
                bool keep = false;
                if (act) {
                    if (!gather) {
                        keep = (__ldg(kbits + (atq[q] >> 5)) >> (atq[q] & 31)) & 1u;
                    } else if ((unsigned)v >= (unsigned long long)n) {
                        atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
                    } else {
                        const int dv = dq[q];
                        keep = (dv > du) || (dv == du && (int64_t)v > u0 + ur);
                    }
                }
                const unsigned km = __ballot_sync(FULL, keep);
                if (!COMPACT && kbits) {
                    // keep bit of entry `at` -> kbits; without hub rows the window
                    // covers 32 consecutive entries, whose bits lane 0 writes as
                    // one word split over the two words it straddles
                    if (hubless) {
                        if (lane == 0 && km) {
                            const long long a0 = atq[q];
                            const int sh = (int)(a0 & 31);
                            atomicOr(kbits + (a0 >> 5), km << sh);
                            if (sh) atomicOr(kbits + (a0 >> 5) + 1, km >> (32 - sh));
                        }
                    } else if (keep) {
                        atomicOr(kbits + (atq[q] >> 5), 1u << (atq[q] & 31));
                    }
                }
                // lanes of this window holding entries of the row of lane `lane`
                const int lo = max(Pex, bw) - bw, hi = min(P, bw + 32) - bw;
                const unsigned rowbits =
                    (lst && lo < hi) ? ((hi >= 32 ? FULL : ((1u << hi) - 1u)) & ~((1u << lo) - 1u)) : 0u;
                if (COMPACT || rdag) {
                    // compaction: the row's next position in dag_col; row-local
                    // count pass: the row's start plus its kept entries so far
                    const int next = __shfl_sync(FULL, cnt, o) + (COMPACT ? 0 : __shfl_sync(FULL, (int)ca, o));
                    const int first = __shfl_sync(FULL, lo, o);  // the row's first lane in the window
                    if (keep) {
                        const long long pos = (long long)next + __popc(km & lt & ~((1u << first) - 1u));
                        if (!COMPACT)
                            rdag[G.ebase + pos] = (int32_t)(vb + v);
                        else if (pos < dag_cap)
                            dag_col[pos] = (int32_t)(vb + v);
                        else
                            atomicOr(&ctr->err, ERRBIT_DAG_OVERFLOW);
                    }
                }
                cnt += __popc(km & rowbits);
            }
        }
        if (!COMPACT && lst) {
            if (bnd) bnd[row0 + rid] = make_int2((int)(G.ebase + ca), cnt);  // row-local DAG: (start, d+)
            else kept[row0 + rid] = cnt;
        }
        if (!COMPACT && rdag) {  // kept entries of the walk, for the symmetry check
            int t = cnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
            if (lane == 0 && t) atomicAdd(reinterpret_cast<unsigned long long*>(&ctr->m), (unsigned long long)t);
        }
    }
}

// Orientation of hub rows (degree > HUB_DEGREE): one block per row, rows
// taken from the hub list with an atomic cursor; then of mid rows
// (MID_DEGREE < degree <= HUB_DEGREE), one warp per row, so that a 32-row
// group of long rows does not hold up a whole orientation pass. A tile is 4 consecutive
// entries per thread (loads issued together); the count pass reduces the
// kept entries of the row, the compaction pass places them in input order
// with a block-wide exclusive scan per tile.
constexpr int HUB_THREADS = 512;

template <typename Off, bool COMPACT, bool BATCH>
__global__ void __launch_bounds__(HUB_THREADS)
    k_orient_hub(GraphRef one, const GraphRef* __restrict__ gs, int k, int64_t total, const int32_t* __restrict__ hubs,
                 const int32_t* __restrict__ deg, int32_t* __restrict__ kept, const int32_t* __restrict__ dag_ptr,
                 int32_t* __restrict__ dag_col, int64_t dag_cap, unsigned* __restrict__ kbits,
                 int32_t* __restrict__ rdag, int2* __restrict__ bnd, DevCounters* ctr) {
    __shared__ int s_row, s_carry;
    __shared__ int s_w[HUB_THREADS / 32];
    if (COMPACT && ctr->err) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = HUB_THREADS / 32;
    const int nh = ctr->n_hub;
    for (;;) {
        if (threadIdx.x == 0) s_row = atomicAdd(&ctr->q_hub[COMPACT ? 1 : 0], 1);
        __syncthreads();
        const int hi = s_row;
        if (hi >= nh) break;
        const int64_t ug = hubs[hi];
        const GraphRef G = graph_of<BATCH>(ug, one, gs, k);
        const int64_t u = ug - G.vbase;
        const Off* rp = static_cast<const Off*>(G.row_ptr);
        const long long a = (long long)rp[u], b = (long long)rp[u + 1];  // checked by k_degree
        const int du = deg[ug];
        const uint64_t pol_stream = l2_policy_first(), pol_keep = l2_policy_last();
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        // output: the compacted DAG, or (row-local count pass) the row itself
        const bool write = COMPACT || rdag;
        int32_t* out = COMPACT ? dag_col : rdag + G.ebase;
        const long long ocap = COMPACT ? dag_cap : 0x7fffffffffffffffLL;
        const int64_t obase = G.vbase;
        long long pos0 = COMPACT ? (long long)dag_ptr[ug] : a;
        int total = 0;
        for (long long t0 = a; t0 < b; t0 += 4LL * HUB_THREADS) {
            const long long e0 = t0 + 4LL * threadIdx.x;
            int v[4], keepc = 0;
            bool kq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = (e0 + q < b) ? ldg_hint(G.col + e0 + q, pol_stream) : -1;
            const bool from_bits = COMPACT && kbits;  // keep decisions of the count pass
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                kq[q] = false;
                if (e0 + q < b) {
                    if (from_bits) {
                        kq[q] = (__ldg(kbits + ((e0 + q) >> 5)) >> ((e0 + q) & 31)) & 1u;
                    } else if ((unsigned)v[q] >= (unsigned long long)G.n) {
                        atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
                    } else {
                        const int dv = ldg_hint(deg + G.vbase + v[q], pol_keep);
                        kq[q] = (dv > du) || (dv == du && (int64_t)v[q] > u);
                    }
                }
                keepc += kq[q];
            }
            if (!COMPACT) total += keepc;
            if (!COMPACT) {
                if (kbits) {
                    // 8 lanes hold 32 consecutive entries as nibbles; the group's
                    // first lane writes them as one word over the two it straddles
                    const unsigned nib = (unsigned)kq[0] | (unsigned)kq[1] << 1 | (unsigned)kq[2] << 2 |
                                         (unsigned)kq[3] << 3;
                    unsigned word = nib << (4 * (lane & 7));
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) word |= __shfl_xor_sync(FULL, word, o);
                    if ((lane & 7) == 0 && word) {
                        const int sh = (int)(e0 & 31);
                        atomicOr(kbits + (e0 >> 5), word << sh);
                        if (sh) atomicOr(kbits + (e0 >> 5) + 1, word >> (32 - sh));
                    }
                }
                if (!write) continue;
            }
            // exclusive block scan of keepc
            int inc = keepc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += t;
            }
            if (lane == 31) s_w[w] = inc;
            __syncthreads();
            if (w == 0) {
                const int x = lane < nw ? s_w[lane] : 0;
                int xi = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FULL, xi, o);
                    if (lane >= o) xi += t;
                }
                if (lane < nw) s_w[lane] = xi - x;
            }
            __syncthreads();
            long long p = pos0 + s_carry + s_w[w] + inc - keepc;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (kq[q]) {
                    if (p < ocap)
                        out[p] = (int32_t)(obase + v[q]);
                    else
                        atomicOr(&ctr->err, ERRBIT_DAG_OVERFLOW);
                    ++p;
                }
            __syncthreads();
            if (threadIdx.x == HUB_THREADS - 1) s_carry += s_w[w] + inc;
            __syncthreads();
        }
        if (!COMPACT) {
            // block sum of the kept entries -> kept[ug]
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(FULL, total, o);
            if (lane == 0) s_w[w] = total;
            __syncthreads();
            if (threadIdx.x == 0) {
                int t = 0;
                for (int i = 0; i < nw; ++i) t += s_w[i];
                if (bnd) bnd[ug] = make_int2((int)(G.ebase + a), t);
                else kept[ug] = t;
                if (rdag && t) atomicAdd(reinterpret_cast<unsigned long long*>(&ctr->m), (unsigned long long)t);
            }
        }
        __syncthreads();
    }
    // mid rows (MID_DEGREE < degree <= HUB_DEGREE): one warp each, taken from
    // the back of the list with an atomic cursor, 64 entries per step
    const int nmid = ctr->n_mid;
    const unsigned lt = (1u << lane) - 1u;
    for (;;) {
        int mi = 0;
        if (lane == 0) mi = atomicAdd(&ctr->q_mid[COMPACT ? 1 : 0], 1);
        mi = __shfl_sync(FULL, mi, 0);
        if (mi >= nmid) break;
        const int64_t ug = hubs[total - 1 - mi];
        const GraphRef G = graph_of<BATCH>(ug, one, gs, k);
        const int64_t u = ug - G.vbase;
        const Off* rp = static_cast<const Off*>(G.row_ptr);
        const long long ra = (long long)rp[u];  // checked by k_degree
        const int rl = (int)((long long)rp[u + 1] - ra);
        int rc = COMPACT ? dag_ptr[ug] : 0;  // compaction: next output position; count: kept so far
        for (int b = 0; b < rl; b += 64) {
            const int f0 = b + lane, f1 = b + 32 + lane;
            const int v0 = f0 < rl ? __ldg(G.col + ra + f0) : -1;
            const int v1 = f1 < rl ? __ldg(G.col + ra + f1) : -1;
            bool k0 = false, k1 = false;
            if (COMPACT && kbits) {
                if (f0 < rl) k0 = (__ldg(kbits + ((ra + f0) >> 5)) >> ((ra + f0) & 31)) & 1u;
                if (f1 < rl) k1 = (__ldg(kbits + ((ra + f1) >> 5)) >> ((ra + f1) & 31)) & 1u;
            } else {
                const bool ok0 = (unsigned)v0 < (unsigned long long)G.n, ok1 = (unsigned)v1 < (unsigned long long)G.n;
                const int d0 = ok0 ? __ldg(deg + G.vbase + v0) : 0;
                const int d1 = ok1 ? __ldg(deg + G.vbase + v1) : 0;
                if ((f0 < rl && !ok0) || (f1 < rl && !ok1)) atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
                k0 = ok0 && ((d0 > rl) || (d0 == rl && (int64_t)v0 > u));
                k1 = ok1 && ((d1 > rl) || (d1 == rl && (int64_t)v1 > u));
            }
            const unsigned km0 = __ballot_sync(FULL, k0), km1 = __ballot_sync(FULL, k1);
            if (!COMPACT && kbits && lane == 0) {
                // 64 consecutive entries from ra + b: bits km0, then km1
                const long long a0 = ra + b;
                const int sh = (int)(a0 & 31);
                unsigned* wd = kbits + (a0 >> 5);
                if (sh == 0) {
                    if (km0) atomicOr(wd, km0);
                    if (km1) atomicOr(wd + 1, km1);
                } else {
                    if (km0 << sh) atomicOr(wd, km0 << sh);
                    if ((km0 >> (32 - sh)) | (km1 << sh)) atomicOr(wd + 1, (km0 >> (32 - sh)) | (km1 << sh));
                    if (km1 >> (32 - sh)) atomicOr(wd + 2, km1 >> (32 - sh));
                }
            }
            if (COMPACT || rdag) {
                const long long rb = COMPACT ? (long long)rc : ra + rc;  // next position of the row's output
                const long long p0 = rb + __popc(km0 & lt);
                const long long p1 = rb + __popc(km0) + __popc(km1 & lt);
                if (!COMPACT) {
                    if (k0) rdag[G.ebase + p0] = (int32_t)(G.vbase + v0);
                    if (k1) rdag[G.ebase + p1] = (int32_t)(G.vbase + v1);
                } else {
                    if (k0) {
                        if (p0 < dag_cap) dag_col[p0] = (int32_t)(G.vbase + v0);
                        else atomicOr(&ctr->err, ERRBIT_DAG_OVERFLOW);
                    }
                    if (k1) {
                        if (p1 < dag_cap) dag_col[p1] = (int32_t)(G.vbase + v1);
                        else atomicOr(&ctr->err, ERRBIT_DAG_OVERFLOW);
                    }
                }
            }
            rc += __popc(km0) + __popc(km1);
        }
        if (!COMPACT && lane == 0) {
            if (bnd) bnd[ug] = make_int2((int)(G.ebase + ra), rc);
            else kept[ug] = rc;
            if (rdag && rc) atomicAdd(reinterpret_cast<unsigned long long*>(&ctr->m), (unsigned long long)rc);
        }
    }
}

// ---- exclusive scan of int32 counts with an int64 carry ---------------------

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 8192
constexpr int SCAN_TOP_THREADS = 1024;

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive block scan; returns the exclusive prefix, *total = block sum.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sh, long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long inc = warp_incl_scan(v, lane);
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        const long long x = (lane < nw) ? sh[lane] : 0;
        const long long xi = warp_incl_scan(x, lane);
        if (lane < nw) sh[lane] = xi - x;
        if (lane == 31) sh[32] = xi;
    }
    __syncthreads();
    const long long r = sh[w] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_reduce(const int32_t* __restrict__ in, int64_t n, long long* __restrict__ partial) {
    __shared__ long long sh[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const int64_t k = base + i;
        if (k < n) s += in[k];
    }
    long long tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// to_warp_count: 1, the scan is of the ordered warp list's key histogram, whose
// total is the warp list's length; 2, of the ordered work items' key
// histogram (the total, the item count, is known already); 0, the DAG
// offsets (total = m).
__global__ void __launch_bounds__(SCAN_TOP_THREADS)
    k_scan_top(long long* __restrict__ partial, int nb, int32_t* __restrict__ out, int64_t n, DevCounters* ctr,
               int to_warp_count) {
    __shared__ long long sh[33];
    const int per = (nb + SCAN_TOP_THREADS - 1) / SCAN_TOP_THREADS;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    long long s = 0;
    for (int i = b0; i < b1; ++i) s += partial[i];
    long long tot;
    long long pre = block_excl_scan(s, sh, &tot);
    for (int i = b0; i < b1; ++i) {
        const long long x = partial[i];
        partial[i] = pre;
        pre += x;
    }
    if (threadIdx.x == 0) {
        if (to_warp_count == 1) {
            ctr->n_warp = (int)tot;  // <= n < 2^31
        } else if (to_warp_count == 0) {
            ctr->m = tot;
            if (tot > 0x7fffffffLL) atomicOr(&ctr->err, ERRBIT_DAG_TOO_BIG);
            out[n] = (int32_t)tot;
        }
    }
}

__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_down(const int32_t* in, int64_t n, const long long* __restrict__ partial, int32_t* out) {
    // in and out may be the same array (the ordered warp list scans in place):
    // a block reads its whole tile before it writes any of it
    __shared__ int s_tile[SCAN_TILE];
    __shared__ long long sh[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const int64_t k = base + i;
        s_tile[i] = (k < n) ? in[k] : 0;
    }
    __syncthreads();
    int* mine = s_tile + threadIdx.x * SCAN_ITEMS;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) s += mine[i];
    long long tot;
    long long pre = block_excl_scan(s, sh, &tot) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int x = mine[i];
        mine[i] = (int)pre;  // exceeds int32 only when ERRBIT_DAG_TOO_BIG is raised
        pre += x;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const int64_t k = base + i;
        if (k < n) out[k] = s_tile[i];
    }
}

// ---- binning ----------------------------------------------------------------

// ncol != nullptr (ordered warp list; ncol: the input CSR's neighbour ids,
// whose rows start where the row-local DAG's do, or a compact DAG's own
// lists): instead of appending a warp-class vertex to the warp list, give it
// the locality key min(u, first entry of its row) -- with sorted rows the
// smallest id of {u} + N(u) (row-local) or {u} + N+(u) (compact DAG), a
// min-hash of the neighbourhood -- in okey[u] and count it in ohist[key];
// k_place then lays the list out in key order.
__global__ void k_bin(const int32_t* __restrict__ dag_ptr, const int2* __restrict__ dag_bnd, int64_t n,
                      int warp_max, int item_nbrs, int shard_count, int shard_index, int32_t* __restrict__ warp_list,
                      int2* __restrict__ warp_desc, int2* __restrict__ items, int64_t item_cap, long long max_m,
                      const int32_t* __restrict__ ncol, int32_t* __restrict__ okey, int32_t* __restrict__ ohist,
                      DevCounters* ctr) {
    if (ctr->err) return;
    if (max_m >= 0 && ctr->m > max_m) {  // more kept entries than an undirected CSR can give
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctr->err, ERRBIT_DAG_OVERFLOW);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t u = base + threadIdx.x;
        int d = 0, a = 0;
        if (u < n && (shard_count <= 1 || (int)(u % shard_count) == shard_index)) {
            if (dag_bnd) {
                const int2 b = dag_bnd[u];
                a = b.x;
                d = b.y;
            } else {
                a = dag_ptr[u];
                d = dag_ptr[u + 1] - a;
            }
        }
        const bool is_warp = d >= 2 && d <= warp_max;
        if (ncol) {
            if (is_warp) {  // d+ >= 2: the row is not empty
                const int c = __ldg(ncol + a);
                const int key = ((unsigned)c < (unsigned long long)u) ? c : (int)u;
                okey[u] = key;
                atomicAdd(&ohist[key], 1);
            }
        } else if (const unsigned wm = __ballot_sync(FULL, is_warp)) {
            const int leader = __ffs(wm) - 1;
            int pos = 0;
            if (lane == leader) pos = atomicAdd(&ctr->n_warp, __popc(wm));
            pos = __shfl_sync(FULL, pos, leader);
            if (is_warp) {
                const int at = pos + __popc(wm & lanemask_lt(lane));
                warp_list[at] = (int32_t)u;
                warp_desc[at] = make_int2(a, d);
            }
        }
        if (d > warp_max) {
            const int k = (d + item_nbrs - 1) / item_nbrs;
            atomicAdd(&ctr->n_block, 1);
            const int pos = atomicAdd(&ctr->n_items, k);
            if ((int64_t)pos + k <= item_cap) {
                for (int j = 0; j < k; ++j) items[pos + j] = make_int2((int)u, j * item_nbrs);
            } else {
                atomicOr(&ctr->err, ERRBIT_DAG_OVERFLOW);
            }
        }
    }
}

// Ordered work items: the key of item i (u, first out-neighbour index j) is the
// id of N+(u)[j], counted into the (zeroed) histogram; items2 holds the items
// as binning wrote them.
__global__ void k_item_key(const int32_t* __restrict__ dag_ptr, const int2* __restrict__ dag_bnd,
                           const int32_t* __restrict__ dcol, const int2* __restrict__ items2, int32_t* __restrict__ ikey,
                           int32_t* __restrict__ ohist, int64_t n, DevCounters* ctr) {
    if (ctr->err) return;
    const int ni = ctr->n_items;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
        const int2 it = items2[i];
        const int a = dag_bnd ? dag_bnd[it.x].x : dag_ptr[it.x];
        int key = __ldg(dcol + a + it.y);
        if ((unsigned)key >= (unsigned long long)n) key = 0;  // a bad id is reported by the counting kernels
        ikey[i] = key;
        atomicAdd(&ohist[key], 1);
    }
}

// Ordered work items, placement: item i takes the next slot of its key's run.
__global__ void k_item_place(const int2* __restrict__ items2, const int32_t* __restrict__ ikey,
                             int32_t* __restrict__ ohist, int2* __restrict__ items, DevCounters* ctr) {
    if (ctr->err) return;
    const int ni = ctr->n_items;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x)
        items[atomicAdd(&ohist[ikey[i]], 1)] = items2[i];
}

// Ordered warp list, second pass: every warp-class vertex takes the next slot
// of its key's run (ohist: the runs' exclusive offsets after the scan), so
// vertices with the same key sit next to each other in the list and are
// counted at about the same time; their out-neighbours overlap, so the 2-hop
// lists they read are shared in L2. The order within a run is arbitrary.
__global__ void k_place(const int32_t* __restrict__ dag_ptr, const int2* __restrict__ dag_bnd, int64_t n,
                        int warp_max, int shard_count, int shard_index,
                        const int32_t* __restrict__ okey, int32_t* __restrict__ ohist, int32_t* __restrict__ warp_list,
                        int2* __restrict__ warp_desc, DevCounters* ctr) {
    if (ctr->err) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        if (shard_count > 1 && (int)(u % shard_count) != shard_index) continue;
        const int2 b = dag_bnd ? dag_bnd[u] : make_int2(dag_ptr[u], dag_ptr[u + 1] - dag_ptr[u]);
        if (b.y >= 2 && b.y <= warp_max) {
            const int pos = atomicAdd(&ohist[okey[u]], 1);
            warp_list[pos] = (int32_t)u;
            warp_desc[pos] = b;
        }
    }
}

template <typename Off, bool BATCH>
cudaError_t orient_t(const GraphRef& one, const GraphRef* gs, int k, int64_t total, int32_t* deg, int32_t* kept,
                     long long* partial, int32_t* dag_ptr, int32_t* dag_col, int64_t dag_cap, int32_t* hubs,
                     unsigned* kbits, int64_t kbits_words, int2* bnd, int32_t* rdag, long long entries,
                     DevCounters* ctr, int num_sms, cudaStream_t st, long long* launches) {
    if (total <= 0) return cudaSuccess;
    if (rdag) kbits = nullptr;  // the row-local DAG needs no compaction pass
    if (kbits) {
        const cudaError_t e = cudaMemsetAsync(kbits, 0, (size_t)kbits_words * 4, st);
        if (e != cudaSuccess) return e;
    }
    *launches += rdag ? 3 : 8;
    const int hg = num_sms * 2;
    const int64_t groups = (total + 31) / 32;
    int og = (int)((groups + ORIENT_WARPS - 1) / ORIENT_WARPS);
    const int og_cap = num_sms * 8 * 4;
    if (og > og_cap) og = og_cap;
    int dg = (int)((total + 255) / 256);
    if (dg > num_sms * 16) dg = num_sms * 16;
    k_degree<Off, BATCH><<<dg, 256, 0, st>>>(one, gs, k, total, deg, hubs, bnd, entries, ctr);
    k_orient<Off, false, BATCH><<<og, ORIENT_THREADS, 0, st>>>(one, gs, k, total, deg, kept, nullptr, nullptr, 0,
                                                                kbits, rdag, bnd, 0, groups, ctr);
    k_orient_hub<Off, false, BATCH><<<hg, HUB_THREADS, 0, st>>>(one, gs, k, total, hubs, deg, kept, nullptr, nullptr, 0,
                                                                 kbits, rdag, bnd, ctr);
    if (rdag) return cudaGetLastError();  // row-local DAG: bnd and rdag are the DAG
    const int nb = scan_blocks(total);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(kept, total, partial);
    k_scan_top<<<1, SCAN_TOP_THREADS, 0, st>>>(partial, nb, dag_ptr, total, ctr, 0);
    k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(kept, total, partial, dag_ptr);
    k_orient<Off, true, BATCH><<<og, ORIENT_THREADS, 0, st>>>(one, gs, k, total, deg, nullptr, dag_ptr, dag_col,
                                                               dag_cap, kbits, nullptr, nullptr, 0, groups, ctr);
    k_orient_hub<Off, true, BATCH><<<hg, HUB_THREADS, 0, st>>>(one, gs, k, total, hubs, deg, nullptr, dag_ptr, dag_col,
                                                                dag_cap, kbits, nullptr, nullptr, ctr);
    return cudaGetLastError();
}

}  // namespace

int scan_blocks(int64_t n) { return (int)((n + SCAN_TILE - 1) / SCAN_TILE); }

cudaError_t launch_orient(const void* row_ptr, int offset_bits, const int32_t* col, int64_t n, int64_t nnz,
                          int32_t* deg, int32_t* kept, long long* partial, int32_t* dag_ptr, int32_t* dag_col,
                          int64_t dag_cap, int32_t* hubs, unsigned* kbits, DevCounters* ctr, int num_sms,
                          cudaStream_t st, long long* launches, int2* bnd, int32_t* rdag) {
    const GraphRef one{row_ptr, col, n, nnz, 0, 0};
    const int64_t words = keep_bits_words(nnz);
    if (offset_bits == 64)
        return orient_t<long long, false>(one, nullptr, 1, n, deg, kept, partial, dag_ptr, dag_col, dag_cap, hubs,
                                          kbits, words, bnd, rdag, nnz, ctr, num_sms, st, launches);
    return orient_t<int32_t, false>(one, nullptr, 1, n, deg, kept, partial, dag_ptr, dag_col, dag_cap, hubs, kbits,
                                    words, bnd, rdag, nnz, ctr, num_sms, st, launches);
}

template <typename Off>
cudaError_t orient_pieces_t(const GraphRef& one, int32_t* deg, int32_t* kept, int32_t* hubs, int2* bnd, int32_t* rdag,
                            DevCounters* ctr, int num_sms, cudaStream_t st, long long* launches,
                            const int64_t* group_cuts, int pieces, const cudaEvent_t* ready) {
    const int64_t total = one.n;
    if (total <= 0) return cudaSuccess;
    int dg = (int)((total + 255) / 256);
    if (dg > num_sms * 16) dg = num_sms * 16;
    k_degree<Off, false><<<dg, 256, 0, st>>>(one, nullptr, 1, total, deg, hubs, bnd, one.nnz, ctr);
    *launches += 2 + pieces;
    for (int i = 0; i < pieces; ++i) {
        cudaError_t e = cudaStreamWaitEvent(st, ready[i], 0);
        if (e != cudaSuccess) return e;
        const int64_t glo = group_cuts[i], ghi = group_cuts[i + 1];
        if (ghi <= glo) continue;
        int og = (int)((ghi - glo + ORIENT_WARPS - 1) / ORIENT_WARPS);
        const int og_cap = num_sms * 8 * 4;
        if (og > og_cap) og = og_cap;
        k_orient<Off, false, false><<<og, ORIENT_THREADS, 0, st>>>(one, nullptr, 1, total, deg, kept, nullptr, nullptr,
                                                                   0, nullptr, rdag, bnd, glo, ghi, ctr);
    }
    k_orient_hub<Off, false, false><<<num_sms * 2, HUB_THREADS, 0, st>>>(one, nullptr, 1, total, hubs, deg, kept,
                                                                       nullptr, nullptr, 0, nullptr, rdag, bnd, ctr);
    return cudaGetLastError();
}

cudaError_t launch_orient_batch(const GraphRef* graphs, int k, int offset_bits, int64_t total, int32_t* deg,
                                int32_t* kept, long long* partial, int32_t* dag_ptr, int32_t* dag_col,
                                int64_t dag_cap, int32_t* hubs, DevCounters* ctr, int num_sms, cudaStream_t st,
                                long long* launches, int2* bnd, int32_t* rdag, long long entries) {
    const GraphRef none{nullptr, nullptr, 0, 0, 0, 0};
    if (offset_bits == 64)
        return orient_t<long long, true>(none, graphs, k, total, deg, kept, partial, dag_ptr, dag_col, dag_cap, hubs,
                                         nullptr, 0, bnd, rdag, entries, ctr, num_sms, st, launches);
    return orient_t<int32_t, true>(none, graphs, k, total, deg, kept, partial, dag_ptr, dag_col, dag_cap, hubs,
                                   nullptr, 0, bnd, rdag, entries, ctr, num_sms, st, launches);
}

cudaError_t launch_orient_row_local_pieces(const void* row_ptr, int offset_bits, const int32_t* col, int64_t n,
                                           int64_t nnz, int32_t* deg, int32_t* kept, int32_t* hubs, int2* bnd,
                                           int32_t* rdag, DevCounters* ctr, int num_sms, cudaStream_t st,
                                           long long* launches, const int64_t* group_cuts, int pieces,
                                           const cudaEvent_t* ready) {
    const GraphRef one{row_ptr, col, n, nnz, 0, 0};
    if (offset_bits == 64)
        return orient_pieces_t<long long>(one, deg, kept, hubs, bnd, rdag, ctr, num_sms, st, launches, group_cuts,
                                          pieces, ready);
    return orient_pieces_t<int32_t>(one, deg, kept, hubs, bnd, rdag, ctr, num_sms, st, launches, group_cuts, pieces,
                                    ready);
}

cudaError_t launch_bin(const int32_t* dag_ptr, int64_t n, const CountCfg& cfg, int32_t* warp_list, int2* warp_desc,
                       int2* items, int64_t item_cap, DevCounters* ctr, int num_sms, cudaStream_t st,
                       long long* launches, const int2* dag_bnd, long long max_m, const int32_t* ncol,
                       int32_t* okey, int32_t* ohist, long long* partial, const int32_t* dcol, int32_t* ikey,
                       int2* items2) {
    if (n <= 0) return cudaSuccess;
    if (!ncol) okey = nullptr;
    const bool order_items = okey && dcol && ikey && items2;
    int2* items_out = items;
    if (order_items) items = items2;  // binning writes here; the placement pass fills items_out
    int g = (int)((n + 255) / 256);
    if (g > num_sms * 16) g = num_sms * 16;
    if (okey) {
        const cudaError_t e = cudaMemsetAsync(ohist, 0, (size_t)n * 4, st);
        if (e != cudaSuccess) return e;
    }
    *launches += okey ? 5 : 1;
    k_bin<<<g, 256, 0, st>>>(dag_ptr, dag_bnd, n, cfg.warp_max_out_degree, cfg.item_neighbors, cfg.shard_count,
                             cfg.shard_index, warp_list, warp_desc, items, item_cap, max_m, okey ? ncol : nullptr,
                             okey, ohist, ctr);
    if (!okey) return cudaGetLastError();
    const int nb = scan_blocks(n);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(ohist, n, partial);
    k_scan_top<<<1, SCAN_TOP_THREADS, 0, st>>>(partial, nb, ohist, n, ctr, 1);
    k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(ohist, n, partial, ohist);
    k_place<<<g, 256, 0, st>>>(dag_ptr, dag_bnd, n, cfg.warp_max_out_degree, cfg.shard_count, cfg.shard_index, okey,
                               ohist, warp_list, warp_desc, ctr);
    if (!order_items) return cudaGetLastError();
    const cudaError_t e = cudaMemsetAsync(ohist, 0, (size_t)n * 4, st);
    if (e != cudaSuccess) return e;
    *launches += 5;
    const int ig = num_sms * 8;
    k_item_key<<<ig, 256, 0, st>>>(dag_ptr, dag_bnd, dcol, items2, ikey, ohist, n, ctr);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(ohist, n, partial);
    k_scan_top<<<1, SCAN_TOP_THREADS, 0, st>>>(partial, nb, ohist, n, ctr, 2);
    k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(ohist, n, partial, ohist);
    k_item_place<<<ig, 256, 0, st>>>(items2, ikey, ohist, items_out, ctr);
    return cudaGetLastError();
}

}  // namespace tcg
