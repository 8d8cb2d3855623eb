// count.cu -- vertex-centric hashed triangle counting on the oriented graph.
//
// TRUST Algorithm 1, run on N+ (Sec. 2.2 orientation; Sec. 3): for every
// vertex u, build a hash table of N+(u) once, then for every v in N+(u) add
// |table ∩ N+(v)|. The pieces, and where they come from:
//   * bucketed table, fixed-size buckets in one contiguous region, slot given
//     by an atomic increment of the bucket's length (Algorithm 1,
//     hashTableConstruction; Sec. 3.1);
//   * hash: multiplicative hashing into B = 2^lgB buckets (Algorithm 1 uses
//     x mod B; see bucket_of for why the GPU tables do not);
//   * a bucket that holds its maximum number of elements is full; further keys
//     go to the next bucket and a search continues through successor buckets
//     while the bucket it scanned was full (Sec. 3.2, last paragraph: linear
//     probing on overflow);
//   * linear search inside a bucket (Algorithm 1, linearSearch);
//   * virtual combination (Sec. 4.2): the 2-hop lists N+(v) of 32
//     out-neighbours are treated as one flat array whose indices are dealt to
//     the 32 lanes; a lane finds the owning list of its index from the
//     inclusive prefix of the list lengths (vc_owner);
//   * degree-aware workers (Sec. 4.3): d+ < 2 is skipped; 2 <= d+ <= T_w goes
//     to warp workers, d+ > T_w to thread-block workers whose out-list is split
//     into work items; both pull work from atomic queues (Sec. 4.3, dynamic
//     assignment);
//   * hits are summed per lane, reduced per warp and block, and added to one
//     uint64 total (Algorithm 1, count +=).
// All tables live entirely in shared memory (sized from d+(u) so that they
// always have room), so the paper's global-memory spill region is not needed.
//
// Warp workers: packs. A single small vertex leaves a warp waiting on a chain
// of dependent global loads (list entry -> out-list -> 2-hop bounds -> 2-hop
// keys) for little work, so a warp takes a *pack* of up to 32 small vertices:
// every vertex gets its own table in the warp's shared-memory area, the
// out-lists of the whole pack are inserted as one flat array, and the 2-hop
// lists of all the pack's out-edges are probed as one virtual combination,
// each lane carrying the table of the edge it came from. Bounds of 2-hop
// lists for chunk c+1 are loaded while chunk c is probed, and every lane
// issues VC_UNROLL independent 2-hop loads before it probes any of them.
//
// Pack table layout. The paper interleaves buckets level-major so that a warp
// scanning one level reads global memory coalesced. A pack table lives in
// shared memory, where each lane reads its own bucket, so a bucket is stored
// whole (bucket-major): PACK_SLOTS = 2 slots = 8 bytes, fetched with one
// vector load and compared without branches. A table for out-degree d+ has
// 8 * nextpow2(d+) slots (at least 4 * min_buckets), i.e. 4 * nextpow2(d+)
// two-slot buckets, so the load factor is <= 1/4 per slot. The per-bucket
// lengths are bytes (4 per word; an atomicAdd of 1 << 8*(h%4) on the word
// claims a slot of bucket h) and live after the slots. A pack whose keys do
// not all fit their home buckets is rebuilt with another hash multiplier, so
// its probes need no overflow chain (k_count_pack).
//
// Thread-block tables use 4-slot (16-byte) buckets, B = 2 * nextpow2(part)
// buckets where that fits the block's budget, else the largest B that fits
// (at most one key per bucket on average), and one 32-bit length word
// per bucket (a bucket of a large table can see more than 255 claims), where
// N+(u) is split into parts of at most P_max keys (the largest power of two
// whose table fits the block's shared memory), each probed by the whole
// 2-hop list: |N+(u) ∩ N+(v)| = sum over parts of |part ∩ N+(v)|. A table in
// which a key missed its home bucket is rebuilt with the next hash multiplier
// (up to BLOCK_REHASH times); probes of an overflow-free table need no chain
// checks. In a table that still overflows, buckets that received more claims
// than slots are marked (mark_overflow), and only a marked bucket sends a
// search on to the next one.
#include <mutex>

#include "tc_internal.h"

namespace tcg {

namespace {

#ifndef VC_UNROLL
#define VC_UNROLL 4
#endif
static_assert(VC_UNROLL == 4, "the bitmap owner path reads four window words at once");

#ifndef PACK_MIN_BLOCKS
#define PACK_MIN_BLOCKS 4
#endif

#ifndef PACK_OCTETS
#define PACK_OCTETS 1  // 1: warp workers read 2-hop lists as 32-byte octets when aligned
#endif
#ifndef OCT_MIN_AVG
#define OCT_MIN_AVG 64  // octets for a chunk whose non-empty 2-hop lists average this many keys
#endif

#ifndef BLOCK_PIECE
#define BLOCK_PIECE 512  // combined 2-hop indices per piece of a thread-block item (fixed pieces)
#endif
#ifndef BLOCK_ADAPTIVE_PIECE
#define BLOCK_ADAPTIVE_PIECE 1  // 1: pieces sized so that each warp of the block gets about two
#endif
#ifndef BLOCK_SLOTS
#define BLOCK_SLOTS 4  // slots per bucket of the thread-block tables (2: overflow chains at load 1/2 cost more)
#endif
#ifndef BLOCK_OVF
#define BLOCK_OVF 1  // 1: thread-block tables mark overflowed buckets; only those send a search on
#endif
#ifndef BLOCK_OCTETS
#define BLOCK_OCTETS 1  // 1: thread-block workers read 2-hop lists as 32-byte octets when dag_col is 32-byte aligned
#endif
#ifndef BLOCK_REHASH
#define BLOCK_REHASH 3  // rebuilds of a thread-block table with a displaced key, each with the next hash multiplier (0..3)
#endif
#ifndef BLOCK_FILTER
#define BLOCK_FILTER 1  // 1: overflow-free thread-block tables keep a 32-bit key signature per bucket, probed first
#endif
#ifndef BLOCK_SPREAD
#define BLOCK_SPREAD 2  // thread-block tables: B = BLOCK_SPREAD * nextpow2(part) buckets when that fits the budget
#endif

// Dynamic shared memory of the counting kernels. The device helpers index
// this array with int offsets (shared-space addressing) instead of taking
// generic pointers into it, so that no access has to convert a generic
// address to a shared one.
extern __shared__ int g_smem[];

constexpr int STAGE_INTS = 224;        // warp workers: 4 x 32 compaction lanes | 32 slot hits | 64-word bitmap
constexpr int BLOCK_STAGE_INTS = 128;  // thread-block workers: 4 x 32 compaction lanes
constexpr int EMPTY = -1;        // an unused slot (vertex ids are >= 0)
constexpr int NOKEY = -2;        // the key of a lane with nothing to probe
// Bit 31 of a bucket's last slot marks an overflowed bucket of a thread-block
// table (mark_overflow). A marked slot holds key | OVF_BIT <= -2 for a vertex
// id key <= 2^31 - 2, so it never equals EMPTY or a key.
constexpr int OVF_BIT = (int)0x80000000u;

__device__ __forceinline__ unsigned lanemask_le(int lane) { return (2u << lane) - 1u; }
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Slots of a group of W <= 8 consecutive dag_col entries that belong to a
// list: with the list at [x0 + lo, x0 + hi) relative to the group's first
// entry x0, bit j is set iff lo <= j < hi. Computed once per group, so the
// group's slots are all probed without per-slot range tests and the hits
// are counted as popc(match bits & mask).
template <int W>
__device__ __forceinline__ unsigned slot_mask(int lo, int hi) {
    const unsigned a = (unsigned)min(max(lo, 0), W), b = (unsigned)min(max(hi, 0), W);
    return (((1u << b) - 1u) >> a) << a;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Virtual-combination index map (Sec. 4.2). Lists live one per lane with
// inclusive prefix P and exclusive prefix Pex; `listlane` marks the lanes
// that hold lists. For the window of flat indices [b, b+32), returns the
// owner list of index b + lane:
//   j0 + popc(starts & lanemask_le(lane)) - (bit 0 of starts),
// j0 = number of lists ending at or before b, bit x of `starts` set iff a
// list starts at b + x (one REDUX.OR). Valid when no empty list starts
// strictly inside the window (lists are compacted, or empty only before it).
__device__ __forceinline__ int vc_owner(int b, int P, int Pex, bool listlane, unsigned le) {
    const int j0 = __popc(__ballot_sync(FULL, listlane && P <= b));
    // 1 << x for 0 <= x < 32, else 0 (the clamped funnel shift drops the bit)
    const unsigned bit = listlane ? __funnelshift_lc(0u, 1u, (unsigned)(Pex - b)) : 0u;
    const unsigned starts = __reduce_or_sync(FULL, bit);
    return j0 + __popc(starts & le) - (int)(starts & 1u);
}

// ---- bucket hash ----------------------------------------------------------------

// Bucket of key w in a table of 2^lgB buckets: the top lgB bits of w times
// 2^32/phi (multiplicative hashing). Algorithm 1 hashes x mod B; vertex ids
// of skewed graphs have biased low bits (an R-MAT id bit is 1 with
// probability ~0.24), so x mod B crowds a hub's neighbours into few buckets
// and probes walk long overflow chains -- the collisions the paper reduces by
// reordering ids (Sec. 4.1). The multiplicative hash spreads any id set
// evenly; the count does not depend on the hash.
// HM = 1 selects Algorithm 1's own hash, x mod B. `mult` is the odd
// multiplier of the multiplicative hash (a pack may switch to another one
// to make its tables overflow-free, see k_count_pack).
constexpr unsigned kHashMult0 = 0x9E3779B1u;  // 2^32 / golden ratio
__device__ __forceinline__ unsigned hash_mult(int i) {
    return i == 0 ? kHashMult0 : i == 1 ? 0x85EBCA77u : i == 2 ? 0xC2B2AE3Du : 0x27D4EB2Fu;
}

template <int HM>
__device__ __forceinline__ int bucket_of(int w, int lgB, unsigned mult = kHashMult0) {
    if (HM == 1) return w & ((1 << lgB) - 1);
    return (int)(((unsigned)w * mult) >> (32 - lgB));
}

// Signature bit of key w in a table of 2^lgB buckets (lgB <= 27): with the
// multiplicative hash h = w * mult, the five hash bits below the bucket bits,
// r = (h >> (27 - lgB)) mod 32, minus one (mod 32) -- the bit that a right
// rotation of the signature word by r brings to bit 31 (vc_range_oct_sig);
// with x mod B, the five id bits above the bucket bits. A bucket's signature
// word has the bits of its keys, so a key whose bit is clear in its home
// bucket's word is not in the bucket.
template <int HM>
__device__ __forceinline__ int sig_bit(int w, int lgB, unsigned mult) {
    if (HM == 1) return (int)(((unsigned)w >> lgB) & 31u);
    return (int)(((((unsigned)w * mult) >> (27 - lgB)) + 31u) & 31u);
}

// ---- table builds (bucket-major buckets of SL slots) ------------------------

// Algorithm 1 hashTableConstruction, one key: claim a slot of bucket h with
// an atomic add on its length byte; a full bucket (SL claims) sends the key
// to the next bucket. sm: shared array; tab/lenw: int offsets of the slots and
// of the length words; B = 2^lgB. Lengths count claims (<= keys <= 255).
// Returns 1 when the key did not fit its home bucket (the table overflowed).
template <int HM, int SL = 4>
__device__ __forceinline__ int insert_b4(int tab, int lenw, int lgB, int w, unsigned mult) {
    const int mask = (1 << lgB) - 1;
    int h = bucket_of<HM>(w, lgB, mult);
    for (int s = 0; s <= mask; ++s) {
        const int sh = 8 * (h & 3);
        const unsigned old = atomicAdd(reinterpret_cast<unsigned*>(g_smem + lenw + (h >> 2)), 1u << sh);
        const int slot = (old >> sh) & 0xff;
        if (slot < SL) {
            g_smem[tab + SL * h + slot] = w;
            return s > 0;
        }
        h = (h + 1) & mask;
    }
    return 1;
}

// Same claim with one 32-bit length word per bucket (thread-block tables,
// whose buckets can see more than 255 claims).
// With SL = 2 the lengths are 16-bit, two per word (a part holds at most
// 2^16 - 1 keys, so a length never carries into its neighbour).
// Returns 1 when the key did not fit its home bucket.
template <int HM, int SL = 4>
__device__ __forceinline__ int insert_b4w(int tab, int lenw, int lgB, int w, unsigned mult) {
    const int mask = (1 << lgB) - 1;
    int h = bucket_of<HM>(w, lgB, mult);
    for (int s = 0; s <= mask; ++s) {
        int slot;
        if (SL == 4) {
            slot = atomicAdd(g_smem + lenw + h, 1);
        } else {
            const int sh = 16 * (h & 1);
            slot = (int)((atomicAdd(reinterpret_cast<unsigned*>(g_smem + lenw + (h >> 1)), 1u << sh) >> sh) & 0xffffu);
        }
        if (slot < SL) {
            g_smem[tab + SL * h + slot] = w;
            return s > 0;
        }
        h = (h + 1) & mask;
    }
    return 1;
}

__device__ __forceinline__ int match4(const int4 q, int w) { return (q.x == w) | (q.y == w) | (q.z == w) | (q.w == w); }

// A bucket of SL slots (4: one 16-byte load; 2: one 8-byte load). A warp's
// shared loads are served in phases of 8 (16-byte) or 16 (8-byte) lanes, and
// lanes of one phase that hit different buckets in the same banks conflict:
// with random buckets, 8-byte buckets cost about two thirds of the shared
// wavefronts of 16-byte buckets per probe.
template <int SL>
struct Bucket;
template <>
struct Bucket<4> {
    int4 q;
    __device__ __forceinline__ static Bucket at(int tab, int h) {
        return {*reinterpret_cast<const int4*>(g_smem + tab + 4 * h)};
    }
    __device__ __forceinline__ int match(int w) const { return match4(q, w); }
    __device__ __forceinline__ bool full() const { return q.w != EMPTY; }
    // overflow-marked tables (see mark_overflow): the last slot may carry OVF_BIT
    __device__ __forceinline__ int match_ovf(int w) const {
        return (q.x == w) | (q.y == w) | (q.z == w) | ((q.w & ~OVF_BIT) == w);
    }
    __device__ __forceinline__ bool overflowed() const { return q.w < EMPTY; }
};
template <>
struct Bucket<2> {
    int2 q;
    __device__ __forceinline__ static Bucket at(int tab, int h) {
        return {*reinterpret_cast<const int2*>(g_smem + tab + 2 * h)};
    }
    __device__ __forceinline__ int match(int w) const { return (q.x == w) | (q.y == w); }
    __device__ __forceinline__ bool full() const { return q.y != EMPTY; }
    __device__ __forceinline__ int match_ovf(int w) const { return (q.x == w) | ((q.y & ~OVF_BIT) == w); }
    __device__ __forceinline__ bool overflowed() const { return q.y < EMPTY; }
};

// Whether a search for a key absent from bucket b must go on to the next
// bucket. Plain tables (OVF = false): b is full (some key of this home may
// have been sent on). Overflow-marked tables (OVF = true): b received more
// claims than it has slots, which mark_overflow records in b's last slot --
// a bucket that is merely full sends nothing on, so its misses stop there.
template <int SL, bool OVF>
__device__ __forceinline__ int bucket_match(const Bucket<SL>& b, int w) {
    return OVF ? b.match_ovf(w) : b.match(w);
}
template <int SL, bool OVF>
__device__ __forceinline__ bool bucket_more(const Bucket<SL>& b) {
    return OVF ? b.overflowed() : b.full();
}

// Algorithm 1 linearSearch continued past bucket h0 (slow path): the
// successor buckets in order, while bucket_more says a key may lie further on.
template <int SL, bool OVF = false>
__device__ __noinline__ int probe_chain(int tab, int mask, int h0, int w) {
    int h = (h0 + 1) & mask;
    for (int s = 0; s < mask; ++s) {
        const Bucket<SL> b = Bucket<SL>::at(tab, h);
        const int hit = bucket_match<SL, OVF>(b, w);
        if (hit | !bucket_more<SL, OVF>(b)) return hit;
        h = (h + 1) & mask;
    }
    return 0;
}

// The next step of a search for w whose home bucket h0 may have sent it on:
// bucket h0 + 1, inline; only a search that must go further calls probe_chain.
template <int SL, bool OVF>
__device__ __forceinline__ int probe_next(int tab, int mask, int h0, int w) {
    const int h = (h0 + 1) & mask;
    const Bucket<SL> b = Bucket<SL>::at(tab, h);
    const int hit = bucket_match<SL, OVF>(b, w);
    if (hit | !bucket_more<SL, OVF>(b)) return hit;
    return probe_chain<SL, OVF>(tab, mask, h, w);
}

// After a thread-block table is built: mark every bucket that received more
// claims than its SL slots -- a key that hashed there was sent to a later
// bucket -- by setting OVF_BIT in its last slot (which holds a key, the
// bucket being full). Claims are the bucket's length counter (32-bit words
// for SL = 4, 16-bit halves for SL = 2). Called by all threads of the block
// between two barriers.
template <int SL>
__device__ __forceinline__ void mark_overflow(int tab, int lenw, int nbuckets) {
    for (int t = threadIdx.x; t < nbuckets; t += blockDim.x) {
        const int claims =
            SL == 4 ? g_smem[lenw + t] : (int)(((unsigned)g_smem[lenw + (t >> 1)] >> (16 * (t & 1))) & 0xffffu);
        if (claims > SL) g_smem[tab + SL * t + SL - 1] |= OVF_BIT;
    }
}

// VC_UNROLL probes per lane: key[q] against the table at int offset kt[q]
// with log2 B = km[q] & 0xffff (pack slot km[q] >> 16). A probe is one
// vector load of the bucket (SL slots) and SL compares; only a lane whose
// bucket may send the key on (bucket_more) and did not match walks the
// overflow chain. NOKEY lanes never match.
template <bool SLOT_HITS, int HM, int SL, bool OVF>
__device__ __forceinline__ uint32_t probe4(const int (&key)[VC_UNROLL], const int (&kt)[VC_UNROLL],
                                           const int (&km)[VC_UNROLL], int stage, unsigned mult) {
    uint32_t hits = 0;
#pragma unroll
    for (int q = 0; q < VC_UNROLL; ++q) {
        const int lg = km[q] & 0xffff;
        const int h = bucket_of<HM>(key[q], lg, mult);
        const Bucket<SL> b = Bucket<SL>::at(kt[q], h);
        int hit = bucket_match<SL, OVF>(b, key[q]);
        const bool more = key[q] >= 0 && !hit && bucket_more<SL, OVF>(b);
        if (__any_sync(FULL, more)) {
            if (more) hit = probe_chain<SL, OVF>(kt[q], (1 << lg) - 1, h, key[q]);
        }
        hits += hit;
        if (SLOT_HITS && hit) atomicAdd(&g_smem[stage + 128 + (km[q] >> 16)], 1);
    }
    return hits;
}

// Probe the 2-hop lists of up to 32 out-edges against bucketed tables.
// Lane i brings the list N+(v_i) = dag_col[s, s+l) and the table of its edge
// (tab: int offset of the slots, lgB = log2 B, slot: pack slot). Empty lists
// are compacted away (stage: STAGE_INTS ints of smem), the rest are combined
// virtually, and the combined indices [skip, min(limit, total)) are dealt out
// 32 at a time, VC_UNROLL windows per step with all loads of a step issued
// before its probes. A probe is one bucket load and SL compares; only a
// lane whose bucket is full and did not match walks the overflow chain.
// Returns the hits; *done = number of combined indices processed.
template <bool SLOT_HITS, int HM, int SL = 4, bool OVF = false>
__device__ __forceinline__ uint32_t vc_range_b4(int s, int l, int tab, int lgB, int slot, int skip, int limit,
                                                const int32_t* __restrict__ dag_col, int lane,
                                                int stage, int* done, unsigned mult = kHashMult0) {
    const unsigned nem = __ballot_sync(FULL, l > 0);
    if (nem == 0) {
        *done = 0;
        return 0;
    }
    const int c = __popc(nem);
    if (l > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = l;
        g_smem[stage + 64 + p] = tab;
        g_smem[stage + 96 + p] = lgB | (slot << 16);
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int cl = lst ? g_smem[stage + 32 + lane] : 0;
    const int ctab = g_smem[stage + 64 + (lst ? lane : 0)];  // lanes past the lists alias list 0's table
    const int cms = lst ? g_smem[stage + 96 + lane] : 0;
    __syncwarp();
    const int P = warp_incl_scan(cl, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int end = total < limit ? total : limit;
    const int Pex = P - cl;
    const int bias = cs - Pex;  // dag_col index of combined position f of this list: bias + f
    const unsigned le = lanemask_le(lane);
    uint32_t hits = 0;
    for (int base = skip; base < end; base += 32 * VC_UNROLL) {
        int key[VC_UNROLL], kt[VC_UNROLL], km[VC_UNROLL];
#pragma unroll
        for (int q = 0; q < VC_UNROLL; ++q) {
            const int b = base + 32 * q;
            const int o = vc_owner(b, P, Pex, lst, le) & 31;
            const int bo = __shfl_sync(FULL, bias, o);
            kt[q] = __shfl_sync(FULL, ctab, o);
            km[q] = __shfl_sync(FULL, cms, o);
            const int f = b + lane;
            key[q] = (f < end) ? __ldg(dag_col + bo + f) : NOKEY;
        }
        hits += probe4<SLOT_HITS, HM, SL, OVF>(key, kt, km, stage, mult);
    }
    *done = end > skip ? end - skip : 0;
    return hits;
}

// Fast probe of whole 2-hop lists against overflow-free pack tables: every
// key is in its home bucket, so one bucket load and SL compares decide it.
// Lane i brings N+(v_i) = dag_col[s, s+l) and its table descriptor
// td = slots offset | log2 B << 16 | pack slot << 21. Owners of flat indices
// come from a bitmap of list starts (bit f set iff a list starts at combined
// index f) when the combined length fits BITMAP_BITS: owner of f = (number of
// starts <= f) - 1, one shared load and two popcounts per window; longer
// chunks use vc_owner.
constexpr int BITMAP_WORDS = 64;  // 2048 combined indices
template <bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t vc_pack_fast(int s, int l, int td,
                                                 const int32_t* __restrict__ dag_col, int lane, int stage,
                                                 unsigned mult) {
    const unsigned nem = __ballot_sync(FULL, l > 0);
    if (nem == 0) return 0;
    const int c = __popc(nem);
    if (l > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = l;
        g_smem[stage + 64 + p] = td;
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int cl = lst ? g_smem[stage + 32 + lane] : 0;
    const int ctd = g_smem[stage + 64 + (lst ? lane : 0)];  // lanes past the lists alias list 0's table
    __syncwarp();
    const int P = warp_incl_scan(cl, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int Pex = P - cl;
    const int bias = cs - Pex;
    const unsigned le = lanemask_le(lane);
    uint32_t hits = 0;
    unsigned* bm = reinterpret_cast<unsigned*>(g_smem + stage + 160);
    const bool use_bm = total <= 32 * BITMAP_WORDS;
    if (use_bm) {
        bm[lane] = 0u;
        bm[lane + 32] = 0u;
        __syncwarp();
        if (lst) atomicOr(&bm[Pex >> 5], 1u << (Pex & 31));
        __syncwarp();
    }
    int cum = 0;  // list starts before the current step (bitmap path)
    for (int base = 0; base < total; base += 32 * VC_UNROLL) {
        int key[VC_UNROLL], kd[VC_UNROLL];
        uint4 words = make_uint4(0u, 0u, 0u, 0u);
        if (use_bm) words = *reinterpret_cast<const uint4*>(bm + (base >> 5));
        const unsigned wq[4] = {words.x, words.y, words.z, words.w};
#pragma unroll
        for (int q = 0; q < VC_UNROLL; ++q) {
            const int b = base + 32 * q;
            int o;
            if (use_bm) {
                o = (cum + __popc(wq[q] & le) - 1) & 31;
                cum += __popc(wq[q]);
            } else {
                o = vc_owner(b, P, Pex, lst, le) & 31;
            }
            const int bo = __shfl_sync(FULL, bias, o);
            kd[q] = __shfl_sync(FULL, ctd, o);
            const int f = b + lane;
            key[q] = (f < total) ? __ldg(dag_col + bo + f) : NOKEY;
        }
#pragma unroll
        for (int q = 0; q < VC_UNROLL; ++q) {
            const int h = bucket_of<HM>(key[q], (kd[q] >> 16) & 31, mult);
            const int hit = Bucket<SL>::at(kd[q] & 0xffff, h).match(key[q]);
            hits += hit;
            if (SLOT_HITS && hit) atomicAdd(&g_smem[stage + 128 + ((kd[q] >> 21) & 31)], 1);
        }
    }
    return hits;
}

// Quad-vectorised variant of vc_pack_fast. The 2-hop lists are read as
// aligned 16-byte quads of dag_col: list [s, e) covers the quads
// [s >> 2, (e + 3) >> 2), the quads of all lists are combined virtually and
// dealt one per lane, so each lane loads four keys with one 16-byte load and
// a warp reads 512 contiguous bytes of a long list; the slots of a quad that
// lie outside [s, e) are masked. This divides the owner search, the two
// shuffles and the address arithmetic of a probe by up to four. dag_col must
// be 16-byte aligned; m = dag_ptr[n] is the number of readable entries, and a
// quad that reaches past it is read entry by entry. Owners: bitmap of list
// starts in quad space when the lists span <= BITMAP_WORDS * 32 quads, else
// vc_owner.
constexpr int QUAD_UNROLL = 2;  // quads in flight per lane
template <bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t vc_pack_quad(int s, int l, int td,
                                                 const int32_t* __restrict__ dag_col, int m, int lane, int stage,
                                                 unsigned mult) {
    const unsigned nem = __ballot_sync(FULL, l > 0);
    if (nem == 0) return 0;
    const int c = __popc(nem);
    if (l > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = s + l;
        g_smem[stage + 64 + p] = td;
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int ce = lst ? g_smem[stage + 32 + lane] : 0;
    const int ctd = g_smem[stage + 64 + (lst ? lane : 0)];  // lanes past the lists alias list 0's table
    __syncwarp();
    const int nq = lst ? ((ce + 3) >> 2) - (cs >> 2) : 0;
    const int P = warp_incl_scan(nq, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int Pex = P - nq;
    const int qbias = (cs >> 2) - Pex;  // global quad index of combined quad f of this list: qbias + f
    const unsigned le = lanemask_le(lane);
    uint32_t hits = 0;
    unsigned* bm = reinterpret_cast<unsigned*>(g_smem + stage + 160);
    const bool use_bm = total <= 32 * BITMAP_WORDS;
    if (use_bm) {
        bm[lane] = 0u;
        bm[lane + 32] = 0u;
        __syncwarp();
        if (lst) atomicOr(&bm[Pex >> 5], 1u << (Pex & 31));
        __syncwarp();
    }
    const int4* __restrict__ quads = reinterpret_cast<const int4*>(dag_col);
    int cum = 0;
    // per-vertex hits (SLOT_HITS): a lane's quads come from lists in list
    // order, so its pack slot only grows; hits are summed per run of one slot
    // and added to the slot's counter when the run ends
    int run_slot = 0, run_hits = 0;
    for (int base = 0; base < total; base += 32 * QUAD_UNROLL) {
        int4 v[QUAD_UNROLL];
        int lo[QUAD_UNROLL], hi[QUAD_UNROLL], kd[QUAD_UNROLL];
        uint2 words = make_uint2(0u, 0u);
        if (use_bm) words = *reinterpret_cast<const uint2*>(bm + (base >> 5));
        const unsigned wq[2] = {words.x, words.y};
#pragma unroll
        for (int q = 0; q < QUAD_UNROLL; ++q) {
            const int b = base + 32 * q;
            int o;
            if (use_bm) {
                o = (cum + __popc(wq[q] & le) - 1) & 31;
                cum += __popc(wq[q]);
            } else {
                o = vc_owner(b, P, Pex, lst, le) & 31;
            }
            const int qb = __shfl_sync(FULL, qbias, o);
            const int so = __shfl_sync(FULL, cs, o);
            const int eo = __shfl_sync(FULL, ce, o);
            kd[q] = __shfl_sync(FULL, ctd, o);
            const int f = b + lane;
            const int x0 = 4 * (qb + f);  // dag_col index of the quad's first slot
            v[q] = make_int4(NOKEY, NOKEY, NOKEY, NOKEY);
            if (f < total) {
                lo[q] = so - x0;
                hi[q] = eo - x0;
                if (x0 + 3 < m) {
                    v[q] = __ldg(quads + (qb + f));
                } else {
                    if (x0 < m) v[q].x = __ldg(dag_col + x0);
                    if (x0 + 1 < m) v[q].y = __ldg(dag_col + x0 + 1);
                    if (x0 + 2 < m) v[q].z = __ldg(dag_col + x0 + 2);
                }
            } else {
                lo[q] = 4;
                hi[q] = 0;
            }
        }
#pragma unroll
        for (int q = 0; q < QUAD_UNROLL; ++q) {
            const int lg = (kd[q] >> 16) & 31;
            const int tab = kd[q] & 0xffff;
            const int key[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
            unsigned mb = 0;  // bit j: slot j matched (every slot is probed; the mask keeps the list's)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int h = bucket_of<HM>(key[j], lg, mult);
                mb |= (unsigned)Bucket<SL>::at(tab, h).match(key[j]) << j;
            }
            const int hq = __popc(mb & slot_mask<4>(lo[q], hi[q]));
            hits += hq;
            if (SLOT_HITS) {
                const int sl = (kd[q] >> 21) & 31;
                if (sl != run_slot) {
                    if (run_hits) atomicAdd(&g_smem[stage + 128 + run_slot], run_hits);
                    run_slot = sl;
                    run_hits = 0;
                }
                run_hits += hq;
            }
        }
    }
    if (SLOT_HITS && run_hits) atomicAdd(&g_smem[stage + 128 + run_slot], run_hits);
    return hits;
}

// 256-bit variant of vc_pack_quad: the 2-hop lists are read as aligned
// 32-byte octets of dag_col (one 256-bit load per lane gives eight keys),
// halving the owner search, shuffles and address arithmetic per key once
// more, at the price of more masked slots at list ends. dag_col must be
// 32-byte aligned; m = readable entries, an octet reaching past it is read
// entry by entry. One octet per lane per step.
struct Octet {
    int v[8];
};
__device__ __forceinline__ Octet ld_octet(const int32_t* p) {
    Octet r;
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
          "=r"(r.v[7])
        : "l"(p));
    return r;
}
template <bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t vc_pack_oct(int s, int l, int td,
                                                const int32_t* __restrict__ dag_col, int m, int lane, int stage,
                                                unsigned mult) {
    const unsigned nem = __ballot_sync(FULL, l > 0);
    if (nem == 0) return 0;
    const int c = __popc(nem);
    if (l > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = s + l;
        g_smem[stage + 64 + p] = td;
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int ce = lst ? g_smem[stage + 32 + lane] : 0;
    const int ctd = g_smem[stage + 64 + (lst ? lane : 0)];  // lanes past the lists alias list 0's table
    __syncwarp();
    const int no = lst ? ((ce + 7) >> 3) - (cs >> 3) : 0;
    const int P = warp_incl_scan(no, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int Pex = P - no;
    const int obias = (cs >> 3) - Pex;  // global octet index of combined octet f of this list: obias + f
    const unsigned le = lanemask_le(lane);
    uint32_t hits = 0;
    unsigned* bm = reinterpret_cast<unsigned*>(g_smem + stage + 160);
    const bool use_bm = total <= 32 * BITMAP_WORDS;
    if (use_bm) {
        bm[lane] = 0u;
        bm[lane + 32] = 0u;
        __syncwarp();
        if (lst) atomicOr(&bm[Pex >> 5], 1u << (Pex & 31));
        __syncwarp();
    }
    int cum = 0;
    int run_slot = 0, run_hits = 0;  // per-vertex hits per run of one pack slot (as in vc_pack_quad)
    // the octet of window base + 32 is loaded while window base is probed;
    // lanes past the combined range keep their last keys with an empty mask
    Octet k, kn;
#pragma unroll
    for (int j = 0; j < 8; ++j) kn.v[j] = NOKEY;
    int lon = 8, hin = 0, kdn = 0;
    auto fetch = [&](int b) {
        int o;
        if (use_bm) {
            const unsigned w0 = bm[b >> 5];
            o = (cum + __popc(w0 & le) - 1) & 31;
            cum += __popc(w0);
        } else {
            o = vc_owner(b, P, Pex, lst, le) & 31;
        }
        const int ob = __shfl_sync(FULL, obias, o);
        const int so = __shfl_sync(FULL, cs, o);
        const int eo = __shfl_sync(FULL, ce, o);
        kdn = __shfl_sync(FULL, ctd, o);
        const int f = b + lane;
        const int x0 = 8 * (ob + f);  // dag_col index of the octet's first slot
        lon = 8;
        hin = 0;
        if (f < total) {
            lon = so - x0;
            hin = eo - x0;
            if (x0 + 7 < m) {
                kn = ld_octet(dag_col + x0);
            } else {
#pragma unroll
                for (int j = 0; j < 7; ++j)
                    if (x0 + j < m) kn.v[j] = __ldg(dag_col + x0 + j);
            }
        }
    };
    if (total > 0) fetch(0);
    for (int base = 0; base < total; base += 32) {
        k = kn;
        const int lo = lon, hi = hin, kd = kdn;
        if (base + 32 < total) fetch(base + 32);
        const int lg = (kd >> 16) & 31;
        const int tab = kd & 0xffff;
        unsigned mb = 0;  // bit j: slot j matched (every slot is probed; the mask keeps the list's)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int h = bucket_of<HM>(k.v[j], lg, mult);
            mb |= (unsigned)Bucket<SL>::at(tab, h).match(k.v[j]) << j;
        }
        const int hq = __popc(mb & slot_mask<8>(lo, hi));
        hits += hq;
        if (SLOT_HITS) {
            const int sl = (kd >> 21) & 31;
            if (sl != run_slot) {
                if (run_hits) atomicAdd(&g_smem[stage + 128 + run_slot], run_hits);
                run_slot = sl;
                run_hits = 0;
            }
            run_hits += hq;
        }
    }
    if (SLOT_HITS && run_hits) atomicAdd(&g_smem[stage + 128 + run_slot], run_hits);
    return hits;
}

// Quad-vectorised variant of vc_range_b4 for one table (thread-block
// workers): lane i brings the list dag_col[s, e) with nq quads; the combined
// quad indices [skip, min(limit, total)) are dealt one per lane, QUAD_UNROLL
// per step; slots outside their list are masked; a key whose bucket is full
// and did not match walks the overflow chain. *done = quads processed.
template <int HM, int SL, bool OVF, bool CHAIN>
__device__ __forceinline__ uint32_t vc_range_quad(int s, int e, int nq, int tab, int lgB, int skip, int limit,
                                                  const int32_t* __restrict__ dag_col, int m, int lane,
                                                  int stage, int* done, unsigned mult) {
    const unsigned nem = __ballot_sync(FULL, nq > 0);
    if (nem == 0) {
        *done = 0;
        return 0;
    }
    const int c = __popc(nem);
    if (nq > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = e;
        g_smem[stage + 64 + p] = nq;
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int ce = lst ? g_smem[stage + 32 + lane] : 0;
    const int cq = lst ? g_smem[stage + 64 + lane] : 0;
    __syncwarp();
    const int P = warp_incl_scan(cq, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int end = total < limit ? total : limit;
    const int Pex = P - cq;
    const int qbias = (cs >> 2) - Pex;
    const unsigned le = lanemask_le(lane);
    const int mask = (1 << lgB) - 1;
    const int4* __restrict__ quads = reinterpret_cast<const int4*>(dag_col);
    uint32_t hits = 0;
    for (int base = skip; base < end; base += 32 * QUAD_UNROLL) {
        int4 v[QUAD_UNROLL];
        int lo[QUAD_UNROLL], hi[QUAD_UNROLL];
#pragma unroll
        for (int q = 0; q < QUAD_UNROLL; ++q) {
            const int b = base + 32 * q;
            const int o = vc_owner(b, P, Pex, lst, le) & 31;
            const int qb = __shfl_sync(FULL, qbias, o);
            const int so = __shfl_sync(FULL, cs, o);
            const int eo = __shfl_sync(FULL, ce, o);
            const int f = b + lane;
            const int x0 = 4 * (qb + f);
            v[q] = make_int4(NOKEY, NOKEY, NOKEY, NOKEY);
            if (f < end) {
                lo[q] = so - x0;
                hi[q] = eo - x0;
                if (x0 + 3 < m) {
                    v[q] = __ldg(quads + (qb + f));
                } else {
                    if (x0 < m) v[q].x = __ldg(dag_col + x0);
                    if (x0 + 1 < m) v[q].y = __ldg(dag_col + x0 + 1);
                    if (x0 + 2 < m) v[q].z = __ldg(dag_col + x0 + 2);
                }
            } else {
                lo[q] = 4;
                hi[q] = 0;
            }
        }
#pragma unroll
        for (int q = 0; q < QUAD_UNROLL; ++q) {
            const int key[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
            int more = 0;  // bit j: slot j's bucket may have sent its key on and did not match
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= lo[q] && j < hi[q]) {
                    const int h = bucket_of<HM>(key[j], lgB, mult);
                    const Bucket<SL> b = Bucket<SL>::at(tab, h);
                    const int hit = bucket_match<SL, OVF>(b, key[j]);
                    hits += hit;
                    if (CHAIN) more |= (!hit && bucket_more<SL, OVF>(b)) << j;
                }
            }
            if (CHAIN && __any_sync(FULL, more)) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((more >> j) & 1)
                        hits += probe_next<SL, OVF>(tab, mask, bucket_of<HM>(key[j], lgB, mult), key[j]);
            }
        }
    }
    *done = end > skip ? end - skip : 0;
    return hits;
}

// Octet variant of vc_range_quad (thread-block workers, dag_col 32-byte
// aligned): lane i brings dag_col[s, e) with no octets (aligned 32-byte
// groups of eight entries); the combined octet indices [skip, min(limit,
// total)) are dealt one per lane per step, each read with one 256-bit load;
// slots outside their list are masked. *done = octets processed.
template <int HM, int SL, bool OVF, bool CHAIN>
__device__ __forceinline__ uint32_t vc_range_oct(int s, int e, int no, int tab, int lgB, int skip, int limit,
                                                 const int32_t* __restrict__ dag_col, int m, int lane,
                                                 int stage, int* done, unsigned mult) {
    const unsigned nem = __ballot_sync(FULL, no > 0);
    if (nem == 0) {
        *done = 0;
        return 0;
    }
    const int c = __popc(nem);
    if (no > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = e;
        g_smem[stage + 64 + p] = no;
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int ce = lst ? g_smem[stage + 32 + lane] : 0;
    const int co = lst ? g_smem[stage + 64 + lane] : 0;
    __syncwarp();
    const int P = warp_incl_scan(co, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int end = total < limit ? total : limit;
    const int Pex = P - co;
    const int obias = (cs >> 3) - Pex;
    const unsigned le = lanemask_le(lane);
    const int mask = (1 << lgB) - 1;
    uint32_t hits = 0;
    for (int base = skip; base < end; base += 32) {
        const int o = vc_owner(base, P, Pex, lst, le) & 31;
        const int ob = __shfl_sync(FULL, obias, o);
        const int so = __shfl_sync(FULL, cs, o);
        const int eo = __shfl_sync(FULL, ce, o);
        const int f = base + lane;
        const int x0 = 8 * (ob + f);  // dag_col index of the octet's first slot
        Octet k;
#pragma unroll
        for (int j = 0; j < 8; ++j) k.v[j] = NOKEY;
        int lo = 8, hi = 0;
        if (f < end) {
            lo = so - x0;
            hi = eo - x0;
            if (x0 + 7 < m) {
                k = ld_octet(dag_col + x0);
            } else {
#pragma unroll
                for (int j = 0; j < 7; ++j)
                    if (x0 + j < m) k.v[j] = __ldg(dag_col + x0 + j);
            }
        }
        int more = 0;  // bit j: slot j's bucket may have sent its key on and did not match
        if constexpr (!CHAIN) {
            // overflow-free table: every slot is probed and the mask keeps the list's
            unsigned mb = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int h = bucket_of<HM>(k.v[j], lgB, mult);
                mb |= (unsigned)bucket_match<SL, OVF>(Bucket<SL>::at(tab, h), k.v[j]) << j;
            }
            hits += __popc(mb & slot_mask<8>(lo, hi));
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= lo && j < hi) {
                    const int h = bucket_of<HM>(k.v[j], lgB, mult);
                    const Bucket<SL> b = Bucket<SL>::at(tab, h);
                    const int hit = bucket_match<SL, OVF>(b, k.v[j]);
                    hits += hit;
                    more |= (!hit && bucket_more<SL, OVF>(b)) << j;
                }
            }
        }
        if (CHAIN && __any_sync(FULL, more)) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if ((more >> j) & 1)
                    hits += probe_next<SL, OVF>(tab, mask, bucket_of<HM>(k.v[j], lgB, mult), k.v[j]);
        }
    }
    *done = end > skip ? end - skip : 0;
    return hits;
}

// Shared-memory word i of the array at shared-window byte address base. The
// address is formed by an integer multiply-add (i * 4 + base) rather than
// the shift-and-add the compiler picks for an indexed load: the probe loop
// below saturates the integer ALU pipe, and the multiply-add issues on the
// FMA pipe (measured: thread-block workers 3 % faster on R-MAT 22 and 24).
__device__ __forceinline__ unsigned lds_word(unsigned i, unsigned base) {
    unsigned v;
    // volatile: the read must stay after the barrier that publishes the words
    asm volatile("{\n\t.reg .b32 a;\n\tmad.lo.u32 a, %1, 4, %2;\n\tld.shared.u32 %0, [a];\n\t}"
                 : "=r"(v)
                 : "r"(i), "r"(base));
    return v;
}

// vc_range_oct for an overflow-free thread-block table with bucket
// signatures (multiplicative hash, 4-slot buckets, int offset sig of the
// signature words), for tables of 2^LGB buckets (LGB = 0: lgB given at run
// time). Every slot reads its signature word: h = w * mult, the bucket is
// h >> (32 - lgB), and a right rotation of the word by h >> (27 - lgB) (the
// rotate takes the amount mod 32) brings the key's signature bit to bit 31,
// which a funnel shift appends to the octet's pass bits. Only the list's
// slots whose bit is set then load their bucket (16 bytes), one set bit per
// round, the key picked from the octet by the bit's index. Lanes past the
// combined range keep their last octet's keys with an empty slot mask.
template <int LGB>
__device__ __forceinline__ uint32_t vc_range_oct_sig(int s, int e, int no, int tab, int lgB_rt, int skip, int limit,
                                                     const int32_t* __restrict__ dag_col, int m, int lane,
                                                     int stage, int* done, unsigned mult, int sig) {
    const int lgB = LGB ? LGB : lgB_rt;
    const unsigned nem = __ballot_sync(FULL, no > 0);
    if (nem == 0) {
        *done = 0;
        return 0;
    }
    const int c = __popc(nem);
    if (no > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        g_smem[stage + p] = s;
        g_smem[stage + 32 + p] = e;
        g_smem[stage + 64 + p] = no;
    }
    __syncwarp();
    const bool lst = lane < c;
    const int cs = lst ? g_smem[stage + lane] : 0;
    const int ce = lst ? g_smem[stage + 32 + lane] : 0;
    const int co = lst ? g_smem[stage + 64 + lane] : 0;
    __syncwarp();
    const int P = warp_incl_scan(co, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int end = total < limit ? total : limit;
    const int Pex = P - co;
    const int obias = (cs >> 3) - Pex;
    const unsigned le = lanemask_le(lane);
    uint32_t hits = 0;
    // the octet of window base + 32 is loaded while window base is probed
    Octet k, kn;
#pragma unroll
    for (int j = 0; j < 8; ++j) kn.v[j] = NOKEY;
    unsigned mskn = 0;
    const unsigned sig_base = (unsigned)__cvta_generic_to_shared(g_smem) + 4u * (unsigned)sig;
    auto fetch = [&](int b) {
        const int o = vc_owner(b, P, Pex, lst, le) & 31;
        const int ob = __shfl_sync(FULL, obias, o);
        const int so = __shfl_sync(FULL, cs, o);
        const int eo = __shfl_sync(FULL, ce, o);
        const int f = b + lane;
        const int x0 = 8 * (ob + f);  // dag_col index of the octet's first slot
        mskn = 0;
        if (f < end) {
            mskn = slot_mask<8>(so - x0, eo - x0);
            if (x0 + 7 < m) {
                kn = ld_octet(dag_col + x0);
            } else {
#pragma unroll
                for (int j = 0; j < 7; ++j)
                    if (x0 + j < m) kn.v[j] = __ldg(dag_col + x0 + j);
            }
        }
    };
    if (skip < end) fetch(skip);
    for (int base = skip; base < end; base += 32) {
        k = kn;
        const unsigned msk = mskn;
        if (base + 32 < end) fetch(base + 32);
        unsigned pass = 0;
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            const unsigned h = (unsigned)k.v[j] * mult;
            const unsigned sw = lds_word(h >> (32 - lgB), sig_base);
            pass = __funnelshift_lc(__funnelshift_r(sw, sw, h >> (27 - lgB)), pass, 1);
        }
        pass &= msk;
        while (pass) {
            const int j = 31 - __clz(pass);
            pass ^= 1u << j;
            const int k01 = (j & 1) ? k.v[1] : k.v[0], k23 = (j & 1) ? k.v[3] : k.v[2];
            const int k45 = (j & 1) ? k.v[5] : k.v[4], k67 = (j & 1) ? k.v[7] : k.v[6];
            const int k03 = (j & 2) ? k23 : k01, k47 = (j & 2) ? k67 : k45;
            const int w = (j & 4) ? k47 : k03;
            hits += Bucket<4>::at(tab, (int)(((unsigned)w * mult) >> (32 - lgB))).match(w);
        }
    }
    *done = end > skip ? end - skip : 0;
    return hits;
}

// ---- intra-vertex workload balancing alternatives (Sec. 4.2) -----------------
// The paper compares virtual combination with three other ways of spreading
// the 2-hop lists N+(v), v in N+(u), over a warp's lanes. They are kept here
// as ablations of the warp workers (tc_params.balance). Each takes the same
// input as vc_pack_quad: lane i holds N+(v_i) = dag_col[s, s + l) and the
// table descriptor td of its out-edge (slots offset | log2 B << 16 | pack
// slot << 21). Every key is probed with probe_one, which follows the
// overflow chain when the home bucket is full and did not match, so the
// count is exact for packs built with or without chains.

template <bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t probe_one(int key, int td, int stage, unsigned mult) {
    if (key < 0) return 0;
    const int lg = (td >> 16) & 31, tab = td & 0xffff;
    const int h = bucket_of<HM>(key, lg, mult);
    const Bucket<SL> b = Bucket<SL>::at(tab, h);
    int hit = b.match(key);
    if (!hit && b.full()) hit = probe_chain<SL>(tab, (1 << lg) - 1, h, key);
    if (SLOT_HITS && hit) atomicAdd(&g_smem[stage + 128 + ((td >> 21) & 31)], 1);
    return (uint32_t)hit;
}

// Warp-centric: the whole warp walks one list at a time, lane j taking
// entries j, j + 32, ...; lanes past the end of a short list idle.
template <bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t balance_wc(int s, int l, int td,
                                               const int32_t* __restrict__ dag_col, int lane, int stage,
                                               unsigned mult) {
    uint32_t hits = 0;
    unsigned lists = __ballot_sync(FULL, l > 0);
    while (lists) {
        const int j = __ffs(lists) - 1;
        lists &= lists - 1;
        const int sj = __shfl_sync(FULL, s, j), lj = __shfl_sync(FULL, l, j), tdj = __shfl_sync(FULL, td, j);
        for (int off = lane; off < lj; off += 32)
            hits += probe_one<SLOT_HITS, HM, SL>(__ldg(dag_col + sj + off), tdj, stage, mult);
    }
    return hits;
}

// Subwarps of S lanes: subwarp g takes the lists of lanes g, g + 32/S, ...,
// one list per round, lane t of the subwarp taking entries t, t + S, ...; a
// round lasts as long as its longest list.
template <int S, bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t balance_sw(int s, int l, int td,
                                               const int32_t* __restrict__ dag_col, int lane, int stage,
                                               unsigned mult) {
    constexpr int G = 32 / S;
    const int g = lane / S, t = lane % S;
    const unsigned ne = __ballot_sync(FULL, l > 0);
    const int last = ne ? 32 - __clz(ne) : 0;  // lanes [0, last) hold all the lists
    uint32_t hits = 0;
    for (int j0 = 0; j0 < last; j0 += G) {
        const int j = j0 + g;  // <= 31: j0 is a multiple of G below 32
        const int sj = __shfl_sync(FULL, s, j), lj = __shfl_sync(FULL, l, j), tdj = __shfl_sync(FULL, td, j);
        const int lmax = (int)__reduce_max_sync(FULL, (unsigned)lj);
        for (int off = t; off < lmax; off += S) {
            const int key = off < lj ? __ldg(dag_col + sj + off) : NOKEY;
            hits += probe_one<SLOT_HITS, HM, SL>(key, tdj, stage, mult);
        }
    }
    return hits;
}

// Physical combination: the lists are copied, one after another with the
// whole warp, into one combined array of (key, table) pairs in this warp's
// device-memory scratch, PC_ROUND entries per round; then every lane walks
// the combined array, entries lane, lane + 32, ... The copy is the cost the
// paper charges to this design.
constexpr int PC_ROUND = 1024;
template <bool SLOT_HITS, int HM, int SL>
__device__ __forceinline__ uint32_t balance_pc(int s, int l, int td,
                                               const int32_t* __restrict__ dag_col, int lane, int stage,
                                               unsigned mult, int2* buf) {
    const int P = warp_incl_scan(l, lane);
    const int total = __shfl_sync(FULL, P, 31);
    const int Pex = P - l;
    uint32_t hits = 0;
    for (int r0 = 0; r0 < total; r0 += PC_ROUND) {
        const int r1 = total - r0 < PC_ROUND ? total : r0 + PC_ROUND;
        unsigned lists = __ballot_sync(FULL, l > 0 && P > r0 && Pex < r1);
        while (lists) {
            const int j = __ffs(lists) - 1;
            lists &= lists - 1;
            const int sj = __shfl_sync(FULL, s, j), pj = __shfl_sync(FULL, P, j);
            const int xj = __shfl_sync(FULL, Pex, j), tdj = __shfl_sync(FULL, td, j);
            const int a = xj > r0 ? xj : r0, b = pj < r1 ? pj : r1;
            for (int f = a + lane; f < b; f += 32) buf[f - r0] = make_int2(__ldg(dag_col + sj + (f - xj)), tdj);
        }
        __syncwarp();
        for (int f = lane; f < r1 - r0; f += 32) {
            const int2 e = buf[f];
            hits += probe_one<SLOT_HITS, HM, SL>(e.x, e.y, stage, mult);
        }
        __syncwarp();
    }
    return hits;
}

// ---- workers -----------------------------------------------------------------

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

// Bounds of N+(v) for an out-neighbour v (0/0 for no neighbour or a bad id).
// dag_bnd: NULL (compact DAG: dag_ptr[v], dag_ptr[v + 1]) or the (start,
// length) pairs of a row-local DAG (one 8-byte load).
__device__ __forceinline__ void list_bounds(int v, const int32_t* __restrict__ dag_ptr,
                                            const int2* __restrict__ dag_bnd, int n, DevCounters* ctr, int& s,
                                            int& l) {
    s = 0;
    l = 0;
    if (v >= 0) {
        if (v < n) {
            if (dag_bnd) {
                const int2 b = __ldg(dag_bnd + v);
                s = b.x;
                l = b.y;
            } else {
                s = __ldg(dag_ptr + v);
                l = __ldg(dag_ptr + v + 1) - s;
            }
        } else {
            atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
        }
    }
}

// Warp workers over packs of small vertices (2 <= d+ <= T_w).
// smem per warp: area[area_ints] | g_smem[stage + STAGE_INTS]. desc[i] = (first
// out-edge, d+) of warp_list[i]. A pack's area holds all its tables' slots
// first, then all their length words.
// BAL: TC_BALANCE_VC (the design) or one of the Sec. 4.2 alternatives above;
// pc_buf: the physical combination's scratch, PC_ROUND pairs per warp.
// OCT: the octet-capable build. With quad == 2 both builds are launched, one
// after the other, and only the one that fits the graph's shape works: the
// octet build when at least 1 % of the counted vertices are thread-block
// vertices (a skewed graph, whose warp workers probe long 2-hop lists), the
// quad build otherwise.
template <bool PER_VERTEX, int HM, int BAL, bool OCT = false>
__global__ void __launch_bounds__(256, PACK_MIN_BLOCKS)
    k_count_pack(const int32_t* __restrict__ dag_ptr, const int32_t* __restrict__ dag_col,
                 const int2* __restrict__ desc, const int32_t* __restrict__ warp_list,
                 unsigned long long* __restrict__ per_vertex, DevCounters* ctr, int n, int area_ints,
                 int lg_min_buckets, int pop, int quad, int timing, const int2* __restrict__ dag_bnd,
                 int2* __restrict__ pc_buf, int strided) {
    if (ctr->err) return;
    if (quad == 2 && (100LL * ctr->n_block >= (long long)ctr->n_warp) != OCT) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = quad ? (dag_bnd ? dag_bnd[n].x : __ldg(dag_ptr + n)) : 0;  // readable dag_col entries
    long long cyc_b = 0, cyc_p = 0;               // build / probe cycles (timing only)
    const unsigned le = lanemask_le(lane);
    const int area = w * (area_ints + STAGE_INTS);  // int offset of this warp's area in smem
    const int stage = area + area_ints;  // int offset of this warp's stage
    const int nlist = ctr->n_warp;
    unsigned long long acc = 0;
    // A pop takes up to `pop` vertices of the warp list, fewer when the list
    // is short, so that there are at least 4 pops per warp of the grid.
    // strided: pop q takes entries q, q + S, q + 2S, ... (S = ceil(nlist /
    // pop)), so every pop is a sample of the whole list and pops cost about
    // the same even when vertex cost follows the list order (R-MAT ids: the
    // heaviest vertices first); else pops take consecutive entries (a batch:
    // the warps then work on a few graphs at a time, whose lists stay in L2).
    {
        const int per = nlist / (4 * (int)(gridDim.x * (blockDim.x >> 5)));
        pop = per < 1 ? 1 : (per < pop ? per : pop);
    }
    const int S = (nlist + pop - 1) / pop;
    for (;;) {
        int i0 = 0;
        if (lane == 0) i0 = atomicAdd(&ctr->q_warp, strided ? 1 : pop);
        i0 = __shfl_sync(FULL, i0, 0);
        if (strided ? i0 >= S : i0 >= nlist) break;
        const int cnt = strided ? min(pop, (nlist - i0 + S - 1) / S) : min(pop, nlist - i0);
        const int li = strided ? i0 + lane * S : i0 + lane;  // this lane's warp-list entry
        int a = 0, k = 0;
        if (lane < cnt) {
            const int2 d = __ldg(desc + li);
            a = d.x;
            k = d.y;
        }
        // 8 * nextpow2(k) slots (at least 4 * min_buckets) in buckets of PACK_SLOTS
        int lgB = 33 - __clz(k > 1 ? k - 1 : 1);  // log2(2 * nextpow2(k))
        lgB = (lgB < lg_min_buckets ? lg_min_buckets : lgB) + (PACK_SLOTS == 2 ? 1 : 0);
        const int B = 1 << lgB;
        const int ftab = (lane < cnt) ? PACK_SLOTS * B : 0, flen = (lane < cnt) ? B / 4 : 0;
        for (int p0 = 0; p0 < cnt;) {
            // the pack: the longest run of vertices from p0 whose tables fit the area
            const int ft = lane >= p0 ? ftab : 0, fl = lane >= p0 ? flen : 0;
            const int FT = warp_incl_scan(ft, lane), FL = warp_incl_scan(fl, lane);
            const bool take = lane >= p0 && lane < cnt && (FT + FL <= area_ints || lane == p0);
            const int p1 = p0 + __popc(__ballot_sync(FULL, take));
            const bool in = lane >= p0 && lane < p1;
            const int tab_used = __shfl_sync(FULL, FT, p1 - 1), len_used = __shfl_sync(FULL, FL, p1 - 1);
            const int my_tab = area + FT - ft;                  // slots of this lane's table
            const int my_len = area + tab_used + FL - fl;       // its length words
            if (PER_VERTEX) g_smem[stage + 128 + lane] = 0;
            // build every table of the pack from the pack's out-lists, one flat
            // array; if any key misses its home bucket, rebuild the pack with the
            // next hash multiplier (up to 4), else probe with overflow chains
            const int kk = in ? k : 0;
            const int K = warp_incl_scan(kk, lane);
            const int Kex = K - kk;
            const int kbias = a - Kex;  // dag_col index of flat out-edge e owned by this lane
            const int E = __shfl_sync(FULL, K, 31);
            const long long t_build = timing ? clock64() : 0;
            unsigned mult = kHashMult0;
            bool chained = false;
            for (int attempt = 0;; ++attempt) {
                for (int t = lane * 4; t < tab_used; t += 128)
                    *reinterpret_cast<int4*>(g_smem + area + t) = make_int4(EMPTY, EMPTY, EMPTY, EMPTY);
                for (int t = lane * 4; t < len_used; t += 128)
                    *reinterpret_cast<int4*>(g_smem + area + tab_used + t) = make_int4(0, 0, 0, 0);
                __syncwarp();
                int ovf = 0;
                for (int b0 = 0; b0 < E; b0 += 32 * VC_UNROLL) {
                    int key[VC_UNROLL], own[VC_UNROLL];
#pragma unroll
                    for (int q = 0; q < VC_UNROLL; ++q) {
                        const int b = b0 + 32 * q;
                        const int o = vc_owner(b, K, Kex, true, le) & 31;
                        const int bo = __shfl_sync(FULL, kbias, o);
                        own[q] = o;
                        key[q] = (b + lane < E) ? __ldg(dag_col + bo + b + lane) : NOKEY;
                    }
#pragma unroll
                    for (int q = 0; q < VC_UNROLL; ++q) {
                        const int tb = __shfl_sync(FULL, my_tab, own[q]);
                        const int lw = __shfl_sync(FULL, my_len, own[q]);
                        const int lg = __shfl_sync(FULL, lgB, own[q]);
                        if (key[q] >= 0) ovf |= insert_b4<HM, PACK_SLOTS>(tb, lw, lg, key[q], mult);
                    }
                }
                __syncwarp();
                if (!__any_sync(FULL, ovf)) break;
                if (HM == 1 || attempt == 3) {
                    chained = true;
                    break;
                }
                mult = hash_mult(attempt + 1);
            }
            const long long t_probe = timing ? clock64() : 0;
            if (timing) cyc_b += t_probe - t_build;
            // probe: chunks of 32 out-edges, bounds of the next chunk prefetched
            uint32_t hits = 0;
            int s = 0, l = 0, etab = 0, elg = 0, eslot = 0;
            {
                const int o = vc_owner(0, K, Kex, true, le) & 31;
                const int bo = __shfl_sync(FULL, kbias, o);
                etab = __shfl_sync(FULL, my_tab, o);
                elg = __shfl_sync(FULL, lgB, o);
                eslot = o;
                list_bounds(lane < E ? __ldg(dag_col + bo + lane) : -1, dag_ptr, dag_bnd, n, ctr, s, l);
            }
            for (int c0 = 0; c0 < E; c0 += 32) {
                int ns = 0, nl = 0, ntab = 0, nlg = 0, nslot = 0;
                if (c0 + 32 < E) {
                    const int o = vc_owner(c0 + 32, K, Kex, true, le) & 31;
                    const int bo = __shfl_sync(FULL, kbias, o);
                    ntab = __shfl_sync(FULL, my_tab, o);
                    nlg = __shfl_sync(FULL, lgB, o);
                    nslot = o;
                    const int e = c0 + 32 + lane;
                    list_bounds(e < E ? __ldg(dag_col + bo + e) : -1, dag_ptr, dag_bnd, n, ctr, ns, nl);
                }
                if (BAL != TC_BALANCE_VC) {
                    const int td = etab | (elg << 16) | (eslot << 21);
                    if (BAL == TC_BALANCE_WC)
                        hits += balance_wc<PER_VERTEX, HM, PACK_SLOTS>(s, l, td, dag_col, lane, stage, mult);
                    else if (BAL == TC_BALANCE_SW8)
                        hits += balance_sw<8, PER_VERTEX, HM, PACK_SLOTS>(s, l, td, dag_col, lane, stage, mult);
                    else if (BAL == TC_BALANCE_SW16)
                        hits += balance_sw<16, PER_VERTEX, HM, PACK_SLOTS>(s, l, td, dag_col, lane, stage, mult);
                    else
                        hits += balance_pc<PER_VERTEX, HM, PACK_SLOTS>(
                            s, l, td, dag_col, lane, stage, mult,
                            pc_buf + ((size_t)blockIdx.x * (blockDim.x >> 5) + w) * PC_ROUND);
                } else if (OCT && !chained && quad == 2 &&
                           __reduce_add_sync(FULL, (unsigned)l) >=
                               (unsigned)OCT_MIN_AVG * __popc(__ballot_sync(FULL, l > 0))) {
                    // octets pay off on long 2-hop lists; on short ones their alignment
                    // and tail slots cost more than the saved owner work (quads below)
                    hits += vc_pack_oct<PER_VERTEX, HM, PACK_SLOTS>(s, l, etab | (elg << 16) | (eslot << 21),
                                                                    dag_col, m, lane, stage, mult);
                } else if (!chained && quad) {
                    hits += vc_pack_quad<PER_VERTEX, HM, PACK_SLOTS>(s, l, etab | (elg << 16) | (eslot << 21), dag_col,
                                                         m, lane, stage, mult);
                } else if (!chained) {
                    hits += vc_pack_fast<PER_VERTEX, HM, PACK_SLOTS>(s, l, etab | (elg << 16) | (eslot << 21), dag_col,
                                                         lane, stage, mult);
                } else {
                    int done;
                    hits += vc_range_b4<PER_VERTEX, HM, PACK_SLOTS>(s, l, etab, elg, eslot, 0, 0x7fffffff, dag_col, lane,
                                                        stage, &done, mult);
                }
                s = ns;
                l = nl;
                etab = ntab;
                elg = nlg;
                eslot = nslot;
            }
            acc += hits;
            if (timing) cyc_p += clock64() - t_probe;
            if (PER_VERTEX) {
                __syncwarp();
                if (in) per_vertex[__ldg(warp_list + li)] = (unsigned long long)g_smem[stage + 128 + lane];
            }
            __syncwarp();
            p0 = p1;
        }
    }
    if (timing && lane == 0) {
        atomicAdd(&ctr->cyc_build, (unsigned long long)cyc_b);
        atomicAdd(&ctr->cyc_probe, (unsigned long long)cyc_p);
    }
    block_add_total(acc, ctr);
}

// Thread-block workers: one block per work item (u, out-neighbours
// [nb0, nb1)) of a vertex with d+ > T_w; nb1 - nb0 <= item_nbrs <= 1024.
// smem: g_smem[stage + nwarps * BLOCK_STAGE_INTS] | S[item_nbrs] | LP[item_nbrs] | table.
// The block loads the item's out-neighbours' list bounds (S = starts, LP =
// inclusive prefix of lengths) once, builds the table of one part of N+(u),
// and its warps take pieces of PIECE combined 2-hop indices from a shared
// counter: a warp finds the list holding its piece's first index by a
// two-round 32-ary search of LP, then probes the piece with the virtual
// combination of the next 32 lists (more rounds if the piece spans more).
template <int PIECE, int HM>
__global__ void __launch_bounds__(1024, 1)
    k_count_block(const int32_t* __restrict__ dag_ptr, const int32_t* __restrict__ dag_col,
                  const int2* __restrict__ items, unsigned long long* __restrict__ per_vertex, DevCounters* ctr,
                  int n, int table_off, int part_max, int item_nbrs, int quad, int timing,
                  const int2* __restrict__ dag_bnd) {
    __shared__ int s_item, s_piece;
    __shared__ int s_wsum[32];
    if (ctr->err) return;
    long long cyc_b = 0, cyc_p = 0;  // build / probe cycles of this warp (timing only)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = quad ? (dag_bnd ? dag_bnd[n].x : __ldg(dag_ptr + n)) : 0;  // readable dag_col entries
    const int stage = w * BLOCK_STAGE_INTS;  // int offset of this warp's stage
    int* S = g_smem + nw * BLOCK_STAGE_INTS;
    int* E = S + item_nbrs;
    int* LP = E + item_nbrs;
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
        const int a = dag_bnd ? dag_bnd[u].x : dag_ptr[u];
        const int k = dag_bnd ? dag_bnd[u].y : dag_ptr[u + 1] - a;
        const int nb0 = item.y, cnt = min(k, nb0 + item_nbrs) - nb0;
        // list bounds of the item's out-neighbours, and the block-wide prefix of their lengths
        int ls = 0, ll = 0;
        if ((int)threadIdx.x < cnt)
            list_bounds(__ldg(dag_col + a + nb0 + threadIdx.x), dag_ptr, dag_bnd, n, ctr, ls, ll);
        // quad path: the prefix counts the quads each list spans
        // quad == 1: the prefix counts the quads each list spans; quad == 2: octets
        const int units = ll <= 0 ? 0
                          : quad == 2 ? ((ls + ll + 7) >> 3) - (ls >> 3)
                          : quad      ? ((ls + ll + 3) >> 2) - (ls >> 2) : ll;
        const int wi = warp_incl_scan(units, lane);
        if (lane == 31) s_wsum[w] = wi;
        __syncthreads();
        if (w == 0) {
            const int x = lane < nw ? s_wsum[lane] : 0;
            s_wsum[lane] = warp_incl_scan(x, lane) - x;
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            S[threadIdx.x] = ls;
            E[threadIdx.x] = ls + ll;
            LP[threadIdx.x] = s_wsum[w] + wi;
        }
        __syncthreads();
        const int W = cnt > 0 ? LP[cnt - 1] : 0;
        uint32_t h = 0;
        for (int p0 = 0; p0 < k && W > 0; p0 += part_max) {
            const int pk = min(part_max, k - p0);
            // 4B slots in buckets of BLOCK_SLOTS, then one length word per 4 slots
            // (32-bit lengths for 4-slot buckets, two 16-bit lengths for 2-slot
            // buckets); at most 1/2 key per 4-slot bucket where the budget allows (such a table is
            // almost always overflow-free after at most one rebuild); the largest
            // parts get the largest table that fits (part_max buckets, up to one key each)
            const int B = min(BLOCK_SPREAD * next_pow2(pk < 32 ? 32 : pk), part_max);
            const int lgB = 31 - __clz(B) + (BLOCK_SLOTS == 2 ? 1 : 0);  // log2 of the bucket count
            const long long t_build = timing ? clock64() : 0;
            int* tab = g_smem + table_off;
            const int lenw = table_off + 4 * B;
            // build; if a key missed its home bucket, rebuild with the next hash
            // multiplier (up to BLOCK_REHASH times) so that every key sits in its
            // home bucket and probes need no overflow chain; a table that still
            // overflows is probed with chains (its overflowed buckets marked)
            unsigned mult = kHashMult0;
            bool chained = false;
            for (int attempt = 0;; ++attempt) {
                for (int t = threadIdx.x * 4; t < 4 * B; t += blockDim.x * 4)
                    *reinterpret_cast<int4*>(tab + t) = make_int4(EMPTY, EMPTY, EMPTY, EMPTY);
                for (int t = threadIdx.x; t < B; t += blockDim.x) g_smem[lenw + t] = 0;
                if (threadIdx.x == 0) s_piece = 0;
                __syncthreads();
                int ovf = 0;
                for (int t = threadIdx.x; t < pk; t += blockDim.x)
                    ovf |= insert_b4w<HM, BLOCK_SLOTS>(table_off, lenw, lgB, __ldg(dag_col + a + p0 + t), mult);
                if (!__syncthreads_or(ovf)) break;
                if (HM == 1 || attempt >= BLOCK_REHASH) {
                    chained = true;
                    if (BLOCK_OVF) {
                        mark_overflow<BLOCK_SLOTS>(table_off, lenw, 1 << lgB);
                        __syncthreads();
                    }
                    break;
                }
                mult = hash_mult(attempt + 1);
            }
            constexpr bool kFilter = BLOCK_FILTER && BLOCK_SLOTS == 4 && HM == 0;  // x mod B tables always chain
            if (kFilter && !chained) {
                // overflow-free: every key sits in its home bucket; the bucket's length
                // word (no longer needed) becomes its signature
                for (int t = threadIdx.x; t < B; t += blockDim.x) {
                    const int4 q = *reinterpret_cast<const int4*>(tab + 4 * t);
                    unsigned sg = 0;
                    if (q.x != EMPTY) sg |= 1u << sig_bit<HM>(q.x, lgB, mult);
                    if (q.y != EMPTY) sg |= 1u << sig_bit<HM>(q.y, lgB, mult);
                    if (q.z != EMPTY) sg |= 1u << sig_bit<HM>(q.z, lgB, mult);
                    if (q.w != EMPTY) sg |= 1u << sig_bit<HM>(q.w, lgB, mult);
                    g_smem[lenw + t] = (int)sg;
                }
                __syncthreads();
            }
            const long long t_probe = timing ? clock64() : 0;
            if (timing) cyc_b += t_probe - t_build;
            // combined units (quads or keys) per piece: about 2 pieces per warp
            // (pieces are equal, so that balances), at least one 32-unit window
            const int unit_min = quad == 2 ? PIECE / 8 : quad ? PIECE / 4 : PIECE;
            int piece = (W + 2 * nw - 1) / (2 * nw);
            piece = BLOCK_ADAPTIVE_PIECE ? (piece < 32 ? 32 : (piece + 31) & ~31) : unit_min;
            for (;;) {
                int pc = 0;
                if (lane == 0) pc = atomicAdd(&s_piece, 1);
                pc = __shfl_sync(FULL, pc, 0);
                int F = pc * piece;
                if (F >= W) break;
                const int F1 = min(W, F + piece);
                while (F < F1) {
                    // j0 = first list with LP[j0] > F (cnt <= 1024: two 32-ary rounds)
                    const int i1 = min(cnt - 1, lane * 32 + 31);
                    const int blk = __popc(__ballot_sync(FULL, lane * 32 < cnt && LP[i1] <= F));
                    const int i2 = blk * 32 + lane;
                    const int j0 = blk * 32 + __popc(__ballot_sync(FULL, i2 < cnt && LP[i2] <= F));
                    const int j = j0 + lane;
                    const int uj = j < cnt ? LP[j] - (j ? LP[j - 1] : 0) : 0;
                    const int sj = j < cnt ? S[j] : 0;
                    const int base_flat = j0 ? LP[j0 - 1] : 0;
                    int done = 0;
                    if (quad == 2) {
                        const int ej = j < cnt ? E[j] : 0;
                        if (kFilter && !chained) {
                            // table sizes 2^6 .. 2^13 buckets with constant shifts
#define TC_OCT_SIG(L)                                                                                       \
    vc_range_oct_sig<L>(sj, ej, uj, table_off, lgB, F - base_flat, F1 - base_flat, dag_col, m, lane, stage, \
                        &done, mult, lenw)
                            switch (lgB) {
                                case 6: h += TC_OCT_SIG(6); break;
                                case 7: h += TC_OCT_SIG(7); break;
                                case 8: h += TC_OCT_SIG(8); break;
                                case 9: h += TC_OCT_SIG(9); break;
                                case 10: h += TC_OCT_SIG(10); break;
                                case 11: h += TC_OCT_SIG(11); break;
                                case 12: h += TC_OCT_SIG(12); break;
                                case 13: h += TC_OCT_SIG(13); break;
                                default: h += TC_OCT_SIG(0); break;
                            }
#undef TC_OCT_SIG
                        } else if (HM == 0 && !chained)  // x mod B tables always chain
                            h += vc_range_oct<HM, BLOCK_SLOTS, false, false>(sj, ej, uj, table_off, lgB,
                                                                             F - base_flat, F1 - base_flat, dag_col,
                                                                             m, lane, stage, &done, mult);
                        else
                            h += vc_range_oct<HM, BLOCK_SLOTS, BLOCK_OVF, true>(sj, ej, uj, table_off, lgB,
                                                                                F - base_flat, F1 - base_flat,
                                                                                dag_col, m, lane, stage, &done, mult);
                    } else if (quad && !chained) {
                        const int ej = j < cnt ? E[j] : 0;
                        h += vc_range_quad<HM, BLOCK_SLOTS, false, false>(sj, ej, uj, table_off, lgB, F - base_flat,
                                                                          F1 - base_flat, dag_col, m, lane,
                                                                          stage, &done, mult);
                    } else if (quad) {
                        const int ej = j < cnt ? E[j] : 0;
                        h += vc_range_quad<HM, BLOCK_SLOTS, BLOCK_OVF, true>(sj, ej, uj, table_off, lgB,
                                                                             F - base_flat, F1 - base_flat,
                                                                             dag_col, m, lane, stage, &done, mult);
                    } else {
                        h += vc_range_b4<false, HM, BLOCK_SLOTS, BLOCK_OVF>(sj, uj, table_off, lgB, 0, F - base_flat,
                                                                            F1 - base_flat, dag_col, lane,
                                                                            stage, &done, mult);
                    }
                    F += done;
                }
            }
            __syncthreads();
            if (timing) cyc_p += clock64() - t_probe;
        }
        acc += h;
        if (per_vertex) {
            const unsigned long long hu = warp_sum_u64(h);
            if (lane == 0 && hu) atomicAdd(&per_vertex[u], hu);
        }
    }
    if (timing && lane == 0) {
        atomicAdd(&ctr->cyc_build, (unsigned long long)cyc_b);
        atomicAdd(&ctr->cyc_probe, (unsigned long long)cyc_p);
    }
    block_add_total(acc, ctr);
}

// Ablation of the edge-centric design (Sec. 3.3, Algorithm 2): a warp takes
// a vertex u and, for every out-edge (u, v), builds the table of N+(u) afresh
// and probes it with N+(v) -- the table is rebuilt d+(u) times instead of
// once. Out-lists longer than the warp's area holds are built part by part,
// each part probed with all of N+(v). Tables have 4-slot buckets with byte
// lengths (insert_b4's layout) and overflow chains; keys are read one per lane.
template <int HM>
__global__ void __launch_bounds__(256) k_count_edge(const int32_t* __restrict__ dag_ptr,
                                                   const int32_t* __restrict__ dag_col,
                                                   unsigned long long* __restrict__ per_vertex, DevCounters* ctr,
                                                   int n, int area_ints, int part_max, int shard_count,
                                                   int shard_index, int timing) {
    if (ctr->err) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int area = w * (area_ints + STAGE_INTS);
    long long cyc_b = 0, cyc_p = 0;
    unsigned long long acc = 0;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(&ctr->q_warp, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= n) break;
        if (shard_count > 1 && u % shard_count != shard_index) continue;
        const int a = dag_ptr[u], k = dag_ptr[u + 1] - a;
        if (k < 2) continue;
        uint32_t hu = 0;
        for (int e = 0; e < k; ++e) {
            int s = 0, l = 0;
            list_bounds(__ldg(dag_col + a + e), dag_ptr, nullptr, n, ctr, s, l);
            for (int p0 = 0; p0 < k; p0 += part_max) {
                const long long t0 = timing ? clock64() : 0;
                const int pk = min(part_max, k - p0);
                int lgB = 33 - __clz(pk > 1 ? pk - 1 : 1);
                lgB = lgB < 4 ? 4 : lgB;
                const int B = 1 << lgB;
                const int tab = area, lenw = area + 4 * B;
                for (int t = lane * 4; t < 4 * B; t += 128)
                    *reinterpret_cast<int4*>(g_smem + tab + t) = make_int4(EMPTY, EMPTY, EMPTY, EMPTY);
                for (int t = lane; t < B / 4; t += 32) g_smem[lenw + t] = 0;
                __syncwarp();
                for (int t = lane; t < pk; t += 32) insert_b4<HM>(tab, lenw, lgB, __ldg(dag_col + a + p0 + t),
                                                                 kHashMult0);
                __syncwarp();
                const long long t1 = timing ? clock64() : 0;
                for (int i = lane; i < l; i += 32) {
                    const int key = __ldg(dag_col + s + i);
                    const int h = bucket_of<HM>(key, lgB);
                    const int4 b4 = *reinterpret_cast<const int4*>(g_smem + tab + 4 * h);
                    int hit = match4(b4, key);
                    if (!hit && b4.w != EMPTY) hit = probe_chain<4>(tab, B - 1, h, key);
                    hu += hit;
                }
                __syncwarp();
                if (timing) {
                    cyc_b += t1 - t0;
                    cyc_p += clock64() - t1;
                }
            }
        }
        acc += hu;
        if (per_vertex) {
            const unsigned long long t = warp_sum_u64(hu);
            if (lane == 0 && t) atomicAdd(&per_vertex[u], t);
        }
    }
    if (timing && lane == 0) {
        atomicAdd(&ctr->cyc_build, (unsigned long long)cyc_b);
        atomicAdd(&ctr->cyc_probe, (unsigned long long)cyc_p);
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

// Collision statistics of 32-bucket tables, one warp per vertex u: per
// bucket, the number of keys of N+(u) it receives (x mod 32, and the top 5
// bits of x * kHashMult0), counted with shared-memory atomics; the largest
// count is u's max collision, and Eq. 2's phi adds the collective out-degree
// of u times it. Launched with 256 threads per block.
__global__ void __launch_bounds__(256) k_collision(const int32_t* __restrict__ dag_ptr,
                                                   const int32_t* __restrict__ dag_col, int64_t n, DevStats* out) {
    __shared__ int cnt[8][2][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    long long mx0 = 0, mx1 = 0;
    unsigned long long phi0 = 0, phi1 = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int a = dag_ptr[u], b = dag_ptr[u + 1];
        if (b == a) continue;
        cnt[wl][0][lane] = 0;
        cnt[wl][1][lane] = 0;
        __syncwarp();
        unsigned long long coll = 0;
        for (int e = a + lane; e < b; e += 32) {
            const int w = dag_col[e];
            coll += (unsigned)(dag_ptr[w + 1] - dag_ptr[w]);
            atomicAdd(&cnt[wl][0][w & 31], 1);
            atomicAdd(&cnt[wl][1][((unsigned)w * kHashMult0) >> 27], 1);
        }
        __syncwarp();
        coll = warp_sum_u64(coll);
        int m0 = cnt[wl][0][lane], m1 = cnt[wl][1][lane];
        __syncwarp();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m0 = max(m0, __shfl_xor_sync(FULL, m0, o));
            m1 = max(m1, __shfl_xor_sync(FULL, m1, o));
        }
        mx0 = max(mx0, (long long)m0);
        mx1 = max(mx1, (long long)m1);
        phi0 += coll * (unsigned)m0;
        phi1 += coll * (unsigned)m1;
    }
    if (lane == 0) {
        atomicMax(&out->maxc[0], mx0);
        atomicMax(&out->maxc[1], mx1);
        atomicAdd(&out->phi[0], phi0);
        atomicAdd(&out->phi[1], phi1);
    }
}

int pack_smem_bytes(const CountCfg& cfg) { return cfg.warps_per_block * (cfg.warp_area_ints + STAGE_INTS) * 4; }

using PackKernel = void (*)(const int32_t*, const int32_t*, const int2*, const int32_t*, unsigned long long*,
                            DevCounters*, int, int, int, int, int, int, const int2*, int2*, int);

// the balance ablations are built for hash_mode 0 only (checked by the parameter resolution)
PackKernel pack_kernel(bool per_vertex, int hm, int bal = TC_BALANCE_VC) {
    switch (bal) {
        case TC_BALANCE_WC:
            return per_vertex ? k_count_pack<true, 0, TC_BALANCE_WC> : k_count_pack<false, 0, TC_BALANCE_WC>;
        case TC_BALANCE_SW8:
            return per_vertex ? k_count_pack<true, 0, TC_BALANCE_SW8> : k_count_pack<false, 0, TC_BALANCE_SW8>;
        case TC_BALANCE_SW16:
            return per_vertex ? k_count_pack<true, 0, TC_BALANCE_SW16> : k_count_pack<false, 0, TC_BALANCE_SW16>;
        case TC_BALANCE_PC:
            return per_vertex ? k_count_pack<true, 0, TC_BALANCE_PC> : k_count_pack<false, 0, TC_BALANCE_PC>;
        default:
            break;
    }
    if (hm == 1) return per_vertex ? k_count_pack<true, 1, TC_BALANCE_VC> : k_count_pack<false, 1, TC_BALANCE_VC>;
    return per_vertex ? k_count_pack<true, 0, TC_BALANCE_VC> : k_count_pack<false, 0, TC_BALANCE_VC>;
}

// the octet-capable build (virtual combination only)
PackKernel pack_kernel_oct(bool per_vertex, int hm) {
    if (hm == 1)
        return per_vertex ? k_count_pack<true, 1, TC_BALANCE_VC, true> : k_count_pack<false, 1, TC_BALANCE_VC, true>;
    return per_vertex ? k_count_pack<true, 0, TC_BALANCE_VC, true> : k_count_pack<false, 0, TC_BALANCE_VC, true>;
}

using BlockKernel = void (*)(const int32_t*, const int32_t*, const int2*, unsigned long long*, DevCounters*, int,
                             int, int, int, int, int, const int2*);

BlockKernel block_kernel(int hm) { return hm == 1 ? k_count_block<BLOCK_PIECE, 1> : k_count_block<BLOCK_PIECE, 0>; }

using EdgeKernel = void (*)(const int32_t*, const int32_t*, unsigned long long*, DevCounters*, int, int, int, int,
                            int, int);

EdgeKernel edge_kernel(int hm) { return hm == 1 ? k_count_edge<1> : k_count_edge<0>; }

// Largest part of N+(u) whose pack table (B = 2 * nextpow2(part) >= 16
// buckets, 4B slots + B/4 byte-length words) fits a warp's area.
int edge_part_max(int area_ints) {
    int p = 1;
    while (true) {
        int b = 2 * next_pow2(2 * p);
        if (b < 16) b = 16;
        if (4 * b + b / 4 > area_ints) break;
        p *= 2;
    }
    return p;
}

int lg2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

}  // namespace

size_t pc_scratch_bytes(const CountCfg& cfg) {
    return (size_t)(cfg.warp_grid > 0 ? cfg.warp_grid : 1) * cfg.warps_per_block * PC_ROUND * sizeof(int2);
}

int pack_table_ints(int max_out_degree, int min_buckets) {
    int b = 2 * next_pow2(max_out_degree < 1 ? 1 : max_out_degree);
    if (b < min_buckets) b = min_buckets;
    const int slots = 4 * b, buckets = slots / PACK_SLOTS;
    return slots + buckets / 4;  // slots, byte lengths
}

// Shared-memory ints a thread-block worker has for its table, after the
// warps' stages and the item's list bounds and prefix.
int count_block_budget_ints(const CountCfg& cfg) {
    return cfg.block_smem_bytes / 4 - (cfg.block_threads / 32) * BLOCK_STAGE_INTS - 3 * cfg.item_neighbors;
}

// Largest part of N+(u) whose thread-block table of B = nextpow2(part) buckets
// (4B slots + B length words) fits the budget; also the most buckets a table has.
int count_block_part_max(const CountCfg& cfg) {
    const int budget = count_block_budget_ints(cfg);
    int p = 32;
    while (5 * (2 * p) <= budget) p *= 2;
    return p;
}

namespace {

// Raise kernel fn's dynamic shared-memory limit on the current device to at
// least `bytes`; a higher limit set before (by another context) is kept.
std::mutex g_smem_limit_mu;
cudaError_t raise_smem_limit(const void* fn, int bytes) {
    std::lock_guard<std::mutex> lk(g_smem_limit_mu);
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) return e;
    if (a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

cudaError_t count_kernel_setup(CountCfg& cfg, int num_sms) {
    const int warp_smem = pack_smem_bytes(cfg);
    cudaError_t e = cudaSuccess;
    for (int pv = 0; pv < 2 && e == cudaSuccess; ++pv) {
        e = raise_smem_limit(reinterpret_cast<const void*>(pack_kernel(pv, cfg.hash_mode, cfg.balance)), warp_smem);
        if (e == cudaSuccess)
            e = raise_smem_limit(reinterpret_cast<const void*>(pack_kernel_oct(pv, cfg.hash_mode)), warp_smem);
    }
    if (e != cudaSuccess) return e;
    e = raise_smem_limit(reinterpret_cast<const void*>(block_kernel(cfg.hash_mode)), cfg.block_smem_bytes);
    if (e != cudaSuccess) return e;
    e = raise_smem_limit(reinterpret_cast<const void*>(edge_kernel(cfg.hash_mode)), warp_smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_kernel(false, cfg.hash_mode, cfg.balance),
                                                      cfg.warps_per_block * 32,
                                                      warp_smem);
    if (e != cudaSuccess) return e;
    cfg.warp_grid = num_sms * (per_sm > 0 ? per_sm : 1);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_kernel(cfg.hash_mode), cfg.block_threads,
                                                      cfg.block_smem_bytes);
    if (e != cudaSuccess) return e;
    cfg.block_grid = num_sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_count(const int32_t* dag_ptr, const int32_t* dag_col, int64_t n, const int32_t* warp_list,
                         const int2* warp_desc, const int2* items, unsigned long long* per_vertex,
                         const CountCfg& cfg, DevCounters* ctr, cudaStream_t st, long long* launches,
                         const int2* dag_bnd, int2* pc_scratch) {
    if (cfg.balance == TC_BALANCE_PC && !pc_scratch) return cudaErrorInvalidValue;
    if (cfg.edge_centric) {
        *launches += 1;
        edge_kernel(cfg.hash_mode)<<<cfg.warp_grid, cfg.warps_per_block * 32, pack_smem_bytes(cfg), st>>>(
            dag_ptr, dag_col, per_vertex, ctr, (int)n, cfg.warp_area_ints, edge_part_max(cfg.warp_area_ints),
            cfg.shard_count, cfg.shard_index, cfg.cycle_timing);
        return cudaGetLastError();
    }
    *launches += 2;
    const int table_off = (cfg.block_threads / 32) * BLOCK_STAGE_INTS + 3 * cfg.item_neighbors;
    const int quad = (cfg.quad_loads && ((uintptr_t)dag_col & 15) == 0) ? 1 : 0;
    // warp workers: with 32-byte aligned lists (PACK_OCTETS, virtual combination)
    // both the quad and the octet-capable builds are launched; the graph's
    // shape, known on the device after binning, picks the one that runs
    const int pack_quad =
        (quad && PACK_OCTETS && cfg.balance == TC_BALANCE_VC && ((uintptr_t)dag_col & 31) == 0) ? 2 : quad;
    // thread-block workers read 32-byte octets when dag_col is 32-byte aligned
    const int block_quad = (quad && BLOCK_OCTETS && ((uintptr_t)dag_col & 31) == 0) ? 2 : quad;
    block_kernel(cfg.hash_mode)<<<cfg.block_grid, cfg.block_threads, cfg.block_smem_bytes, st>>>(
        dag_ptr, dag_col, items, per_vertex, ctr, (int)n, table_off, count_block_part_max(cfg), cfg.item_neighbors,
        block_quad, cfg.cycle_timing, dag_bnd);
    pack_kernel(per_vertex != nullptr, cfg.hash_mode, cfg.balance)<<<cfg.warp_grid, cfg.warps_per_block * 32,
                                                                   pack_smem_bytes(cfg), st>>>(
        dag_ptr, dag_col, warp_desc, warp_list, per_vertex, ctr, (int)n, cfg.warp_area_ints,
        lg2(cfg.warp_min_buckets), cfg.chunk, pack_quad, cfg.cycle_timing, dag_bnd, pc_scratch,
        cfg.pop_contiguous ? 0 : 1);
    if (pack_quad == 2) {
        *launches += 1;
        pack_kernel_oct(per_vertex != nullptr, cfg.hash_mode)<<<cfg.warp_grid, cfg.warps_per_block * 32,
                                                                pack_smem_bytes(cfg), st>>>(
            dag_ptr, dag_col, warp_desc, warp_list, per_vertex, ctr, (int)n, cfg.warp_area_ints,
            lg2(cfg.warp_min_buckets), cfg.chunk, pack_quad, cfg.cycle_timing, dag_bnd, pc_scratch,
            cfg.pop_contiguous ? 0 : 1);
    }
    return cudaGetLastError();
}

cudaError_t launch_finish(const DevCounters* ctr, unsigned long long* count_out, int* err_out, cudaStream_t st,
                          long long* launches) {
    *launches += 1;
    k_finish<<<1, 1, 0, st>>>(ctr, count_out, err_out);
    return cudaGetLastError();
}

cudaError_t launch_stats(const int32_t* dag_ptr, const int32_t* dag_col, int64_t n, int warp_max_out_degree,
                         DevStats* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int g = (int)((n + 255) / 256);
    if (g > 4096) g = 4096;
    k_stats<<<g, 256, 0, st>>>(dag_ptr, dag_col, n, warp_max_out_degree, out);
    k_collision<<<g, 256, 0, st>>>(dag_ptr, dag_col, n, out);
    return cudaGetLastError();
}

}  // namespace tcg
