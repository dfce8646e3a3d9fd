// common.cuh - shared device definitions for the synchronization check kernels.
//
// Items and the per-group summary
// -------------------------------
// An access becomes an item: a 64-bit word (schedule position << 32 | gtid),
// where the schedule position is the visit order (or, for unsorted traces,
// the rank of (visit order, record index)). Items of one group compare by
// schedule position because positions are unique.
//
// Per group and per action category c in {read, write, atomic} the kernels
// keep a "top-2" summary: first[c] = the earliest item, second[c] = the
// earliest item whose owner differs from first[c]'s owner. The summary of a
// union is the summary of the union of the summaries, so groups reduce in any
// order (no stable sort, no ordered scan needed).
//
// Why the summary is enough. Let (p, q) be the lowest conflicting pair of a
// class in a group (q the later access, the pair minimising (q, p)). Suppose q
// is not in the top-2 of its category. Then first and second of that category
// are either both earlier than q with distinct owners, or first is earlier and
// shares q's owner. In both cases some top-2 item c earlier than q has an owner
// different from p's, lies in q's category, and so conflicts with p in the
// same class; the pair (p, c) ends before q, contradicting minimality. The
// same argument applied to p for the fixed q shows p is in the top-2 of its
// category. So the lowest pair of each class is among the pairs drawn from the
// at most six summary items, and whether two epochs' groups hold any
// conflicting pair is likewise decided by their summaries (Theorem 1 and
// Algorithm 5 of the paper, restated over summaries).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace simk {

constexpr uint32_t ACT_R = 0, ACT_W = 1, ACT_A = 2;
constexpr uint32_t TF_UNSORTED = 1, TF_WARP_AWARE = 2, TF_PAPER_ORDER = 4;     // trace flags
constexpr uint32_t STMT_DIVERGED = 0x80000000u;
constexpr uint64_t EMPTY = ~0ull;
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_PASSES = 40;   // sort passes of one call over 8-bit digits (histograms from the record reads)
constexpr int W_PASSES = 64;     // sort passes of one call over digits of another width (own histograms)
constexpr int W_SLOT_PASSES = 11;   // passes of one stream at the narrowest width (64-bit keys, 6 bits)
constexpr int W_RADIX_MAX = 2048;   // digits of the widest width (11 bits)

// One trace of a call (a single-trace call is a batch of one). Device array
// in the workspace, written by the host side of the call.
struct TraceDesc {
    const uint4 *events;       // records of this trace
    const uint32_t *counts;    // barrier counts, nb * bt
    uint64_t n;                // records
    uint64_t rec_off;          // index of this trace's first record in the batch
    uint64_t tile_off;         // first ingest tile of this trace
    uint32_t block_off;        // batch-wide index of this trace's block 0
    uint32_t nb, bt, su, gu, maxb, flags;
    uint32_t hash_ok;          // eligible for the short-interval hash path (host decision)
    uint32_t hlist;            // hash-path traces: position of block 0 in the hash-path block list
    uint64_t sig_off;          // direct signature table: the slot of this trace's unit 0
    const uint32_t *stmt;      // warp-aware traces: statement word per record
    uint8_t *races;    uint64_t races_cap;    // outputs (device), as in simulee_outputs
    uint8_t *divs;     uint64_t divs_cap;
    uint8_t *reds;     uint64_t reds_cap;
    uint32_t *grid;    uint64_t grid_cap;
    uint8_t *report;                          // simulee_report of this trace
};

// Per-trace device state, zeroed by every call.
struct TState {
    unsigned long long bad_rec;   // ~index (in the trace) of the first bad record, 0 = none
    unsigned long long bad_cnt;   // ~index of the first bad barrier count, 0 = none
    unsigned int n_races;         // race records of the trace
    unsigned int n_grid;          // grid-redundant barriers of the trace
    unsigned int race_start;      // position of the trace's first race in the sorted race list
    unsigned int inel;            // hash-path trace whose blocks are not contiguous in record order
};

// Device control block at the start of the workspace; zeroed by every call.
struct Ctl {
    unsigned int timeout;         // a bounded wait gave up
    unsigned int n_s, n_g;        // shared-intra and global-intra stream sizes
    unsigned int n_xf;            // inter-block records left by the block-signature filter
    unsigned int n_races;         // staged race records (all traces)
    unsigned int n_x;             // inter-block records written by the ingest
    unsigned int n_div, n_red;    // divergent blocks / redundant barriers (all traces)
    unsigned int n_q;             // records in the schedule-rank sort (unsorted traces)
    unsigned int n_fb;            // tiles listed for the fallback read
    unsigned int hb_next[4];      // next list entry for the hash path's CTAs, per launch group
    unsigned int n_rf;            // race records left by the race filter
    unsigned int px_tile;         // next tile of the visit-order scan
    unsigned int tiles[MAX_PASSES];  // onesweep tile counters, one per pass
    unsigned int wtiles[W_PASSES];   // the same for passes over digits of another width
    unsigned int rg_tiles[3];        // next tile of the segmented reductions (S, G, X streams)
    unsigned int hb_gbeg[5];         // hash path: first list entry of each launch group, then all entries
};

// Batch-wide dimensions, bit layouts and workspace offsets of one call (host-computed).
struct Layout {
    uint64_t n;                      // records, all traces
    uint32_t T;                      // traces
    uint32_t NB;                     // blocks, all traces
    uint64_t ntiles_in;              // ingest tiles, all traces
    uint32_t maxb;                   // largest max_barriers
    uint32_t any_unsorted;
    uint32_t swords;                 // words per block of the spilled-run bitmap (epochs 0..maxb)
    uint32_t bb, bus, bug, be, bu, btr;   // bit widths: batch block, shared unit, global unit, epoch,
                                           // max(unit), trace index
    uint32_t bits_s, bits_g, bits_x, bits_r, bits_q;
    uint32_t any_paper;              // a trace has the paper's visit-order counters
    uint32_t bxr;                    // bits of the visit-order field of inter-block keys (0 without such a trace)
    uint32_t np_s, np_g, np_x, np_r, np_q;    // radix passes per stream
    uint32_t p0_s, p0_g, p0_x, p0_r, p0_q;    // first pass index of each stream
    uint32_t wide_s, wide_g, wide_x, wide_q;  // 64-bit keys
    uint32_t words;                  // 32-bit words per block in the barrier bitmaps
    uint64_t race_cap;               // staging capacity for race records
    uint64_t status_tiles;           // tiles covered by the look-back status array
    uint32_t sort_items;             // radix-sort tile: 256 threads x this many elements (8 or 16)
    uint32_t radix_bits;             // digit width of the radix passes (6, 8 or 11)
    uint32_t hb_cap_eighths;         // hash path: distinct units a run may hold, in eighths of its table
    uint32_t hb_pool_div;            // hash path: racy units resolved in place per run, table size / this
    size_t off_hw, off_dw;           // histograms and digit bases of passes not 8 bits wide, per stream
    uint64_t rg_tiles;               // tiles of the largest stream a segmented reduction scans
    size_t off_rgpub, off_rgready;   // the reductions' published tile summaries and their ready words
    size_t off_binel;                // per batch-wide block: the hash path does not apply to it
    size_t off_spill;                // per block and epoch: a run the hash path leaves to the sort path
    size_t off_tflag;                // per ingest tile: holds a spilled run
    size_t off_bbins;                // hash-path block sizes: histogram and placement cursors per launch group
    size_t off_bstart;               // per batch-wide block of a hash-path trace: its first record
    size_t off_blist;                // hash-path blocks, grouped by the CTA shape that takes them
    size_t off_bgroup;               // per batch-wide block of a hash-path trace: its launch group (u8)
    size_t off_fbt;                  // tiles for the fallback read
    size_t off_sig;                  // block signature per global unit (or unit hash)
    uint64_t sig_slots;              // entries of the signature table (0: no global memory)
    uint32_t sig_direct;             // the table is indexed by the trace's offset plus the unit
    uint32_t sig_or;                 // signatures are ORs of (block | ~block << 15)
    uint64_t x_cap;                  // elements of the first inter-block stream buffer (every global record)
    uint64_t cap_s;                  // elements of each intra-block stream buffer (S and G)
    uint64_t cap_x1;                 // elements of the second inter-block buffer (kept by the filter)
    uint32_t compact;                // some capacity is below the worst case: counts are checked against them
    size_t off_ctl, off_td, off_ts, off_tob, off_stats, off_nonred, off_gridnr, off_gridhas, off_cnt_div,
        off_cnt_red, off_ofs_div, off_ofs_red, off_hist, off_dbase, off_status, off_rank, off_p2v;
    size_t off_sk[2], off_sv[2], off_gk[2], off_gv[2], off_xk[2], off_xv[2];
    size_t off_rk[2], off_rv[2], off_rp;
    size_t zero_end;                 // bytes from the start that every call zeroes
    size_t total;
};

// 32-bit integer mixer (the finaliser of MurmurHash3)
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- 1-D bulk copies (TMA) into shared memory, completed on an mbarrier --------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order earlier generic-proxy accesses of shared memory before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for phase `parity` of a barrier, giving up after limit_ns of wall time
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0;; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// stop work that depends on sorted data: a wait gave up
__device__ __forceinline__ bool must_stop(const Ctl *ctl) {
    const volatile Ctl *c = ctl;
    return c->timeout != 0;
}

__device__ __forceinline__ bool trace_bad(const TState &t) {
    const volatile TState *v = &t;
    return v->bad_rec != 0 || v->bad_cnt != 0;
}

// index t with key(t) <= x < key(t+1) over T ascending entries (binary search)
template <class F>
__device__ __forceinline__ uint32_t find_trace(uint32_t T, uint64_t x, F key) {
    uint32_t lo = 0, hi = T;   // invariant: key(lo) <= x, answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (key(mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// payload of a stream element: (act << 30 | gtid) << 32 | schedule position
__device__ __forceinline__ uint64_t make_payload(uint32_t act, uint32_t gtid, uint32_t pos) {
    return ((uint64_t)((act << 30) | gtid) << 32) | pos;
}
__device__ __forceinline__ uint32_t payload_act(uint64_t v) { return (uint32_t)(v >> 62); }
// item = position << 32 | gtid
__device__ __forceinline__ uint64_t payload_item(uint64_t v) {
    return ((uint64_t)(uint32_t)v << 32) | ((uint32_t)(v >> 32) & 0x3FFFFFFFu);
}
__device__ __forceinline__ uint32_t item_pos(uint64_t x) { return (uint32_t)(x >> 32); }
__device__ __forceinline__ uint32_t item_gtid(uint64_t x) { return (uint32_t)x; }

// owners: threads (intra-block groups) or blocks (inter-block groups)
struct OwnThread {
    __device__ __forceinline__ uint32_t operator()(uint64_t x) const { return (uint32_t)x; }
};
// Inter-block owners. The inter-block stream codes an access's thread as
// block << 10 | tid when the trace's blocks fit 20 bits (pad), else as
// block * block_threads + tid.
struct OwnBlock {
    uint32_t bt;
    bool pad;
    __device__ __forceinline__ uint32_t operator()(uint64_t x) const {
        return pad ? ((uint32_t)x >> 10) : (uint32_t)x / bt;
    }
    __device__ __forceinline__ uint32_t gtid(uint32_t code) const {
        return pad ? (code >> 10) * bt + (code & 0x3FFu) : code;
    }
};

struct Top2 {
    uint64_t a[3], b[3];   // per category: first, second (EMPTY when absent)
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int c = 0; c < 3; c++) { a[c] = EMPTY; b[c] = EMPTY; }
    }
    __device__ __forceinline__ bool empty() const { return a[0] == EMPTY && a[1] == EMPTY && a[2] == EMPTY; }
};

template <class Own>
__device__ __forceinline__ void top2_insert(uint64_t &a, uint64_t &b, uint64_t x, const Own &own) {
    if (x < a) {
        if (a != EMPTY && own(a) != own(x)) b = a;
        a = x;
    } else if (x != a && own(x) != own(a) && x < b) {
        b = x;
    }
}

template <class Own>
__device__ __forceinline__ void top2_add(Top2 &s, uint32_t act, uint64_t x, const Own &own) {
    if (act == ACT_R) top2_insert(s.a[0], s.b[0], x, own);
    else if (act == ACT_W) top2_insert(s.a[1], s.b[1], x, own);
    else top2_insert(s.a[2], s.b[2], x, own);
}

template <class Own>
__device__ __forceinline__ void top2_merge(Top2 &s, const Top2 &o, const Own &own) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (o.a[c] != EMPTY) top2_insert(s.a[c], s.b[c], o.a[c], own);
        if (o.b[c] != EMPTY) top2_insert(s.a[c], s.b[c], o.b[c], own);
    }
}

// The lowest pair of class cls (0 WW, 1 RW) among summary items.
// Returns false when the group holds no conflicting pair of that class.
template <class Own>
__device__ __forceinline__ bool lowest_pair(const Top2 &s, int cls, const Own &own, uint64_t &p, uint64_t &q) {
    uint64_t bq = EMPTY, bp = EMPTY;
    // candidate list: categories 1 (write) and 2 (atomic) are the modifying ones
    uint64_t it[6] = {s.a[0], s.b[0], s.a[1], s.b[1], s.a[2], s.b[2]};
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = 0; j < 6; j++) {
            if (j <= i) continue;
            const int ci = i >> 1, cj = j >> 1;
            const uint64_t x = it[i], y = it[j];
            if (x == EMPTY || y == EMPTY) continue;
            const bool mi = ci != 0, mj = cj != 0;
            if (!mi && !mj) continue;                 // read & read
            if (ci == 2 && cj == 2) continue;         // atomic & atomic
            const int pc = (mi && mj) ? 0 : 1;
            if (pc != cls) continue;
            if (own(x) == own(y)) continue;
            const uint64_t lo = x < y ? x : y, hi = x < y ? y : x;
            if (hi < bq || (hi == bq && lo < bp)) { bq = hi; bp = lo; }
        }
    }
    if (bq == EMPTY) return false;
    p = bp;
    q = bq;
    return true;
}

// Does any item of summary P conflict with any item of summary Q (owners: threads)?
__device__ __forceinline__ bool any_conflict(const Top2 &P, const Top2 &Q) {
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const uint64_t x = (i & 1) ? P.b[i >> 1] : P.a[i >> 1];
        if (x == EMPTY) continue;
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const uint64_t y = (j & 1) ? Q.b[j >> 1] : Q.a[j >> 1];
            if (y == EMPTY) continue;
            const int ci = i >> 1, cj = j >> 1;
            if (ci == 0 && cj == 0) continue;
            if (ci == 2 && cj == 2) continue;
            if ((uint32_t)x == (uint32_t)y) continue;
            return true;
        }
    }
    return false;
}

}  // namespace simk
