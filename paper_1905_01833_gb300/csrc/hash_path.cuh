// hash_path.cuh - the single-read path: one CTA per block of a trace whose
// records come block by block and, inside a block, epoch by epoch (the order
// Algorithm 3's simulator emits them).
//
// The CTA finds its block's record range (k_block_ranges), then streams the
// range once, two records per thread per window, and for every record:
//   * validates it (the checks of the ingest) and routes a global record to
//     the inter-block stream X, marking the unit's block signature;
//   * inserts it into a shared-memory hash table of the current (block, epoch)
//     run, keyed by (unit, space), whose entry keeps an owner summary per
//     action category {read, write, atomic}: the OR of the thread ids and the
//     OR of their complements (10 bits each). A set of threads is one thread
//     exactly when the two ORs share no bit, and the union of two sets is
//     one thread exactly when the ORs of the union share no bit, so a single
//     atomicOr per record keeps everything the conflict tests need.
// At the end of a run the creator of each entry decides (a) whether the unit
// holds a conflicting pair inside the run (Theorem 1: owners differ, one
// access modifies, not both atomic), and (b) whether it conflicts with the
// same unit in the previous epoch's table (barrier e-1 needed, Algorithm 5's
// adjacency test). For the units of (a) the exact lowest pair of each class
// comes from two atomicMin passes over the run's records into a pool of top-2
// summaries (common.cuh) laid over the previous run's table, which is free
// once the adjacency test is done; a run with more racy units than that pool
// holds (a third of the table's entries) is marked for the sort path instead
// ("spilled"), which then computes its races exactly.
//
// A block falls back to the sort path entirely ("binel") when its records are
// not in epoch order, a run has more distinct units than the table holds, or a
// record of another block or an invalid record lies in its range. Adjacency
// marks the CTA made before that are sound (each comes from a genuine pair of
// the block's records); its emitted races are dropped by the race filter, and
// the fallback read routes the block to the sort path.
#pragma once
#include "check_kernels.cuh"

namespace simk {

// CTA shapes: one CTA of 768 threads per SM with 8192-entry run tables, or
// two CTAs of 512 threads per SM with 4096-entry tables (so that one CTA's
// barriers overlap the other's work). A CTA of the smaller shape may also be
// split into 2 or 4 thread groups, each with its own quarter or half of the
// tables and its own named barrier, checking one block each: blocks whose runs
// are short (a few hundred records) then fill their windows, and a run's
// barriers and finalisation involve only its group's threads.
// A run may hold up to 7/8 of its group's table in distinct units (runs near
// that load are rare and only probe longer; a run beyond it sends its block to
// the sort path); the options of a call may lower that cutover (4/8 to 7/8)
// and the racy-unit pool (table / 3 down to table / 64).
__host__ __device__ constexpr int hb_log2(int x) { return x <= 1 ? 0 : 1 + hb_log2(x / 2); }
template <int THREADS, int SLOTS, int PER, int CTAS, int GROUPS = 1>
struct HbShape {
    static constexpr int threads = THREADS;           // threads of the CTA
    static constexpr int slots = SLOTS;               // table entries of the CTA, all groups
    static constexpr int ctas_per_sm = CTAS;
    static constexpr int groups = GROUPS;             // blocks checked at once by one CTA
    static constexpr int gthreads = THREADS / GROUPS; // threads of a group
    static constexpr int gslots = SLOTS / GROUPS;     // table entries of a group
    static constexpr int per = PER;                   // records per thread per window
    static constexpr int window = PER * gthreads;     // records per window of a group
    static constexpr int cap = gslots / 8 * 7;        // distinct units per run
    static constexpr int shift = 32 - hb_log2(gslots);
    static constexpr int pool = gslots / 3;           // racy units per run (24-byte summaries in 8-byte entries)
    static_assert(THREADS % (32 * GROUPS) == 0 && (gslots & (gslots - 1)) == 0 && GROUPS <= 4, "group shape");
    static_assert((cap + gthreads - 1) / gthreads <= 32, "list entries per thread");
};
// Two records per thread per window: with four per thread and half the threads (the same tables and
// windows, twice the registers per thread) the kernel ran 40% slower, 16 warps per SM hiding too little
// of the shared-memory and global latencies.
// The larger shape has 768 threads (79 registers each) rather than 1024 (64 registers): the batched
// workload's hash stage was 1.3% faster, its 1024-thread blocks' runs still filling 4-5 windows.
using HbLarge = HbShape<768, 8192, 2, 1>;
using HbSmall = HbShape<512, 4096, 2, 2>;
// Thread groups take one record per thread per window: with two, the extra registers of a group's
// addressing spill (64 registers per thread at two 512-thread CTAs per SM) and the batched workload's
// hash stage was 0.7% slower.
using HbHalf = HbShape<512, 4096, 1, 2, 2>;      // two groups of 256 threads, 2048-entry tables
using HbQuarter = HbShape<512, 4096, 1, 2, 4>;   // four groups of 128 threads, 1024-entry tables

// a group's barrier: the CTA barrier for one group, else named barrier 1 + g over the group's warps
// (immediate barrier ids, so that the kernel reserves only the barriers it uses)
template <class SH>
__device__ __forceinline__ void hb_sync() {
    if constexpr (SH::groups == 1) {
        __syncthreads();
    } else {
        switch (threadIdx.x >> hb_log2(SH::gthreads)) {
        case 0: asm volatile("bar.sync 1, %0;" ::"n"(SH::gthreads) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"n"(SH::gthreads) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"n"(SH::gthreads) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"n"(SH::gthreads) : "memory"); break;
        }
    }
}

// per-group scalars; the per-run ones are indexed by the run's table parity: the finalisation of one
// run clears the next run's set, so a run needs no barrier between its finalisation and the next
// run's inserts
struct HbGroupState {
    uint32_t blk, flag, ridx, cnt[2], first[2], nracy[2], needed[2];
};

constexpr uint32_t HB_EMPTY = 0xFFFFFFFFu;
constexpr uint32_t HB_NONE = 0xFFFFFFFFu;           // no epoch
constexpr uint32_t HB_POS_LIMIT = 1u << 22;         // run positions in a pool item (22 bits)
constexpr uint32_t HB_XCH = 256;                    // inter-block slots a warp reserves at a time
constexpr int HB_RM = 4;                            // run records per thread held across the two pool passes

// Shared memory, one region per thread group: owner summaries [2][gslots] (u64), keys [2][gslots] (u32),
// creation lists [2][cap] (u16), the group's scalars. A group addresses everything from one base.
template <class SH>
__host__ __device__ constexpr size_t hb_group_bytes() {
    return ((size_t)SH::gslots * 24 + (size_t)SH::cap * 4 + sizeof(HbGroupState) + 15) / 16 * 16;
}
template <class SH>
constexpr size_t hash_blocks_smem() {
    return (size_t)SH::groups * hb_group_bytes<SH>();
}

// owner summary field of category c: OR(tid) | OR(~tid) << 10
__device__ __forceinline__ uint64_t hb_own_bits(uint32_t cat, uint32_t tid) {
    const uint32_t f = (tid & 0x3FFu) | ((~tid & 0x3FFu) << 10);
    return (uint64_t)f << (20 * cat);
}
__device__ __forceinline__ uint32_t hb_field(uint64_t o, int c) { return (uint32_t)(o >> (20 * c)) & 0xFFFFFu; }
// the union of two owner sets (given by their fields) holds two or more threads
__device__ __forceinline__ bool hb_two(uint32_t f, uint32_t g) {
    const uint32_t u = f | g;
    return (u & (u >> 10) & 0x3FFu) != 0u;
}
// Two non-empty sets X, Y have x in X, y in Y with different owners exactly
// when their union has two owners (if every cross pair shared an owner, X and
// Y would both be that one owner).

// a conflicting pair inside one run's unit
__device__ __forceinline__ bool hb_racy(uint64_t o) {
    const uint32_t r = hb_field(o, 0), w = hb_field(o, 1), a = hb_field(o, 2), m = w | a;
    if (!hb_two(r | m, r | m)) return false;                      // one thread only (the usual case)
    const bool ww = w && (hb_two(w, w) || (a && hb_two(w, a)));   // write-write, write-atomic
    const bool rw = r && m && hb_two(r, m);                       // read with write or atomic
    return ww || rw;
}

// a conflicting pair between epoch e-1 (P) and epoch e (Q) of a unit:
// read x modify, modify x read, write x modify, atomic x write (never read x read, atomic x atomic)
__device__ __forceinline__ bool hb_cross(uint64_t P, uint64_t Q) {
    const uint32_t pr = hb_field(P, 0), pw = hb_field(P, 1), pa = hb_field(P, 2), pm = pw | pa;
    const uint32_t qr = hb_field(Q, 0), qw = hb_field(Q, 1), qa = hb_field(Q, 2), qm = qw | qa;
    if (!hb_two(pr | pm, qr | qm)) return false;                  // one thread only (the usual case)
    return (pr && qm && hb_two(pr, qm)) || (pm && qr && hb_two(pm, qr)) || (pw && qm && hb_two(pw, qm)) ||
           (pa && qw && hb_two(pa, qw));
}

template <class SH>
__device__ __forceinline__ uint32_t hb_hash(uint32_t key) { return (key * 0x9E3779B1u) >> SH::shift; }

// pool item: run position << 10 | tid  ->  summary item: position << 32 | tid
__device__ __forceinline__ uint64_t hb_item64(uint32_t v) {
    return v == HB_EMPTY ? EMPTY : (((uint64_t)(v >> 10) << 32) | (v & 0x3FFu));
}

// ---------------------------------------------------------------------------
// First record of every block of a hash-path trace: the lower bound of the
// block id over the records, by a 32-way search per warp. The result is
// monotone in the block id for any record order, so the ranges partition the
// trace even when it is not block-contiguous (which the hash kernel detects).
//
// The hash kernel's CTAs take blocks from a queue, and a block's records are
// read by one CTA, so a launch lasts at least as long as its largest block. In
// a batch the large blocks lie anywhere in the list (trace order); a CTA that
// takes one late finishes long after the others. The list is therefore put in
// order of decreasing record count (largest first: the classical longest-
// processing-time rule, within about a percent of the balanced load on the
// batched workload, against about 35% above it in trace order for its
// 1024-thread blocks). Sizes are binned by quarter octaves, which is as good
// for the rule and needs no sort: a histogram per launch, then a placement.
// ---------------------------------------------------------------------------
constexpr int HB_BINS = 128;   // block-size bins per launch group

// quarter-octave bin of a record count, non-decreasing in n (0..3 exact, then 4 bins per octave)
__device__ __forceinline__ uint32_t hb_size_bin(uint32_t n) {
    if (n < 4u) return n;
    const uint32_t l = 31u - __clz(n);   // 2..31
    return 4u * l - 4u + ((n >> (l - 2u)) & 3u);
}

// lower bound of block id lb over a trace's records, by one warp (all lanes return it)
__device__ __forceinline__ uint64_t hb_lower_bound(const TraceDesc &d, uint32_t lb, int lane) {
    uint64_t lo = 0, hi = d.n;   // the answer lies in [lo, hi]
    if (lb == 0) return 0;
    while (hi - lo > 32) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = min(lo + (uint64_t)(lane + 1) * step - 1, hi - 1);
        const bool below = d.events[p].z < lb;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, below);
        const int f = __ffs(~m) - 1;   // first probe not below (-1: all below)
        if (f < 0) {
            lo = hi;
        } else {
            const uint64_t pf = min(lo + (uint64_t)(f + 1) * step - 1, hi - 1);
            const uint64_t pl = f > 0 ? min(lo + (uint64_t)f * step - 1, hi - 1) + 1 : lo;
            lo = pl;
            hi = pf;
        }
    }
    const uint64_t p = lo + lane;
    const bool below = p < hi && d.events[p].z < lb;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, below);
    const int f = __ffs(~m) - 1;
    lo = f < 0 ? lo + 32 : lo + f;
    return min(lo, hi);
}

// Launch groups of the hash path, in list order: blocks of the smaller CTA shape checked by groups of
// 128 threads (HB_LG_QUARTER), of 256 threads (HB_LG_HALF) or by whole CTAs (HB_LG_SMALL), then the
// blocks of the larger shape (HB_LG_LARGE). The host puts each trace's blocks in the smaller or the
// larger class (list entries below or above small_end). Inside the smaller class a block goes to the
// smallest group whose table holds each of its runs, found by sampling the epochs of its records every
// `stride` records (a quarter of the distinct units a quarter table may hold): records are in epoch
// order inside a block, and any 4 * stride consecutive records contain four samples, so a run of
// 4 * stride records or more holds two samples three apart, and one of 8 * stride or more two samples
// seven apart. No equal samples three apart: every run is shorter than a quarter table's capacity;
// none seven apart: shorter than a half table's. (A run's distinct units are at most its records.)
// Runs up to 3 * stride (7 * stride) records never show such a pair.
constexpr int HB_LG_QUARTER = 0, HB_LG_HALF = 1, HB_LG_SMALL = 2, HB_LG_LARGE = 3, HB_LGROUPS = 4;

// launch group of a block of the smaller class whose records are [lo, hi), by one warp (all lanes
// return it)
__device__ __forceinline__ uint32_t hb_sampled_group(const uint4 *ev, uint64_t lo, uint64_t hi, uint32_t stride,
                                                     int lane) {
    uint32_t prev = 0x20000u + lane;   // this lane's sample of the previous chunk (none yet: unique)
    bool near3 = false, near7 = false;  // two samples three / seven strides apart in one epoch
    for (uint64_t base = lo; base < hi && !near7; base += 32ull * stride) {
        const uint64_t p = base + (uint64_t)lane * stride;
        const uint32_t ep = p < hi ? (ev[p].w >> 16) & 0xFFFu : 0x10000u + lane;   // past the end: unique
        const uint32_t up3 = __shfl_up_sync(0xFFFFFFFFu, ep, 3), up7 = __shfl_up_sync(0xFFFFFFFFu, ep, 7);
        const uint32_t pc3 = __shfl_sync(0xFFFFFFFFu, prev, (lane + 29) & 31);   // previous chunk, lane + 29
        const uint32_t pc7 = __shfl_sync(0xFFFFFFFFu, prev, (lane + 25) & 31);   // previous chunk, lane + 25
        near3 |= __any_sync(0xFFFFFFFFu, ep == (lane >= 3 ? up3 : pc3));
        near7 |= __any_sync(0xFFFFFFFFu, ep == (lane >= 7 ? up7 : pc7));
        prev = ep;
    }
    return !near3 ? HB_LG_QUARTER : (!near7 ? HB_LG_HALF : HB_LG_SMALL);
}

// bstart and launch group of every hash-path block, and the size histogram of each launch group; hist
// (HB_LGROUPS x HB_BINS) is zeroed by the call
__global__ void k_block_ranges(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, Layout L,
                               uint32_t small_end, uint32_t groups_on, uint32_t *bstart, uint8_t *bgroup,
                               uint32_t *hist) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // a quarter of a quarter table's distinct units at the call's cutover (1024 / 8 * eighths / 4)
    const uint32_t stride = 32u * L.hb_cap_eighths;
    for (uint64_t b = warp; b < L.NB; b += nwarps) {
        const TraceDesc &d = td[tob[b]];
        if (!d.hash_ok) continue;
        const uint32_t lb = (uint32_t)(b - d.block_off);
        const uint64_t lo = hb_lower_bound(d, lb, lane);
        const uint64_t hi = lb + 1 < d.nb ? hb_lower_bound(d, lb + 1, lane) : d.n;
        const uint32_t entry = d.hlist + lb;
        const uint32_t q = entry >= small_end ? (uint32_t)HB_LG_LARGE
                           : !groups_on       ? (uint32_t)HB_LG_SMALL
                                              : hb_sampled_group(d.events, lo, hi, stride, lane);
        if (lane == 0) {
            bstart[b] = (uint32_t)lo;
            bgroup[b] = (uint8_t)q;
            atomicAdd(&hist[q * HB_BINS + hb_size_bin((uint32_t)(hi - lo))], 1u);
        }
    }
}

// Each launch group's list in order of decreasing block size (bins from the largest down; the order
// inside a bin is the order of the placing atomics). hist and bgroup as k_block_ranges left them;
// cursor zeroed; gbeg[q] = first list entry of launch group q (gbeg[HB_LGROUPS] = all entries).
__global__ void k_block_order(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob,
                              const uint32_t *__restrict__ bstart, const uint8_t *__restrict__ bgroup, Layout L,
                              const uint32_t *__restrict__ hist, uint32_t *cursor, uint32_t *gbeg, uint32_t *blist) {
    __shared__ uint32_t base[HB_LGROUPS * HB_BINS];   // first list entry of each (group, bin)
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int q = 0; q < HB_LGROUPS; q++) {
            if (blockIdx.x == 0) gbeg[q] = acc;
            for (int k = HB_BINS - 1; k >= 0; k--) {
                base[q * HB_BINS + k] = acc;
                acc += hist[q * HB_BINS + k];
            }
        }
        if (blockIdx.x == 0) gbeg[HB_LGROUPS] = acc;
    }
    __syncthreads();
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < L.NB; b += (uint64_t)gridDim.x * blockDim.x) {
        const TraceDesc &d = td[tob[b]];
        if (!d.hash_ok) continue;
        const uint32_t lb = (uint32_t)(b - d.block_off);
        const uint32_t s0 = bstart[b], s1 = lb + 1 < d.nb ? bstart[b + 1] : (uint32_t)d.n;
        const uint32_t bin = bgroup[b] * HB_BINS + hb_size_bin(s1 - s0);
        blist[base[bin] + atomicAdd(&cursor[bin], 1u)] = (uint32_t)b;
    }
}

// one unused inter-block slot: key 0 with an invalid action, dropped by the filter
template <class KX>
__device__ __forceinline__ void hb_x_fill(KX *xk, uint64_t *xv, uint32_t from, uint32_t to, uint64_t cap, int lane) {
    for (uint32_t o = from + lane; o < to; o += 32)
        if (o < cap) {
            xk[o] = (KX)0;
            xv[o] = ~0ull;
        }
}

// HOT: a warp marks a global unit's block signature once per run of consecutive lanes holding the same
// unit and block (a unit that every thread reads would otherwise take one atomic per record on one word)
template <class KX, class SH, bool HOT>
__global__ void __launch_bounds__(SH::threads, SH::ctas_per_sm)
k_hash_blocks(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, const uint32_t *__restrict__ bstart,
              const uint32_t *__restrict__ blist, const uint32_t *__restrict__ gbeg, int lgroup,
              const uint4 *__restrict__ stats, unsigned int *queue, Layout L, TState *ts, Ctl *ctl, uint32_t *nonred, uint32_t *binel, uint32_t *spill, uint32_t *tflag,
              KX *xk, uint64_t *xv, uint32_t *sig, RaceStage rs) {
    // this launch's blocks: list entries lbeg .. lbeg + lcnt - 1
    const uint32_t lbeg = gbeg[lgroup], lcnt = gbeg[lgroup + 1] - lbeg;
    if (lcnt == 0) return;
    extern __shared__ __align__(16) uint64_t hb_smem[];
    const int g = SH::groups == 1 ? 0 : (int)(threadIdx.x >> hb_log2(SH::gthreads));
    const int tid = SH::groups == 1 ? (int)threadIdx.x : (int)(threadIdx.x & (SH::gthreads - 1));
    const int lane = threadIdx.x & 31;
    uint8_t *const greg = reinterpret_cast<uint8_t *>(hb_smem) + (size_t)g * hb_group_bytes<SH>();
    uint64_t *own = reinterpret_cast<uint64_t *>(greg);                            // [2][gslots]
    uint32_t *key = reinterpret_cast<uint32_t *>(greg + 16 * SH::gslots);          // [2][gslots]
    uint16_t *list = reinterpret_cast<uint16_t *>(greg + 24 * SH::gslots);         // [2][cap]
    HbGroupState &S = *reinterpret_cast<HbGroupState *>(greg + 24 * SH::gslots + 4 * SH::cap);
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < 2 * SH::gslots; i += SH::gthreads) {
        own[i] = 0ull;
        key[i] = HB_EMPTY;
    }
    if (tid == 0) {
        S.flag = 0;
        S.ridx = 0;
        for (int q = 0; q < 2; q++) {
            S.cnt[q] = 0;
            S.first[q] = HB_NONE;
            S.nracy[q] = 0;
            S.needed[q] = 0;
        }
    }
    const uint64_t xcap = L.x_cap;
    uint32_t xpos = 0, xend = 0;   // this warp's reserved inter-block slots [xpos, xend)
    // the cutover to the sort path chosen for the call: distinct units per run, racy units per run
    const uint32_t cap_rt = min((uint32_t)SH::cap, (uint32_t)SH::gslots / 8u * L.hb_cap_eighths);
    const uint32_t pool_rt = min((uint32_t)SH::pool, (uint32_t)SH::gslots / L.hb_pool_div);
    for (;;) {
        hb_sync<SH>();
        if (tid == 0) S.blk = atomicAdd(queue, 1u);
        hb_sync<SH>();
        if (S.blk >= lcnt) break;
        const uint32_t b = blist[lbeg + S.blk];
        const uint32_t t = tob[b];
        const TraceDesc &d = td[t];
        // uniform: only hash-path traces whose barrier counts are valid (otherwise nothing is reported)
        if (!d.hash_ok || *(volatile unsigned long long *)&ts[t].bad_cnt) continue;
        const uint32_t lb = b - d.block_off;
        const uint32_t s0 = bstart[b], s1 = (lb + 1 < d.nb) ? bstart[b + 1] : (uint32_t)d.n;
        if (s0 >= s1) continue;   // a block without records: no runs
        const uint4 *ev = d.events;
        const uint32_t *cnts = d.counts;
        // the block's smallest barrier count: a record of this block at an epoch up to it is within its
        // thread's count, so only later epochs (diverged threads) need the thread's count
        const uint32_t bmin = stats[b].x;
        const uint32_t nb = d.nb, bt = d.bt, su = d.su, gu = d.gu, maxb = d.maxb;
        const bool pad = nb <= (1u << 20);
        uint32_t *const sig_t = L.sig_direct ? sig + d.sig_off : sig;   // this trace's stretch of a direct table

        // ---- windows: records wbase + j * SH::gthreads + tid, j = 0, 1. A run's first window
        //      starts at the run's first record; records below vmark are already validated and
        //      routed (a window that starts inside the previous one re-reads them from cache).
        uint32_t wbase = s0, vmark = s0;
        constexpr int P = SH::per;
        uint4 cur[P], nxt[P];
        auto load = [&](uint4 (&w)[P], uint32_t base) {
#pragma unroll
            for (int j = 0; j < P; j++) {
                const uint32_t i = base + j * SH::gthreads + tid;
                w[j] = i < s1 ? ev[i] : make_uint4(0, 0, 0, 0);
            }
        };
        // validate the window's new records, route global ones to X; returns the window's
        // records of this block (those to hash)
        auto activate = [&]() -> uint32_t {
            uint32_t pb = 0;
            bool stopme = false, isx[P], same[P];   // same: the lane before holds this record's unit and block
#pragma unroll
            for (int j = 0; j < P; j++) {
                const uint32_t idx = wbase + j * SH::gthreads + tid;
                const bool in = idx < s1, fresh = in && idx >= vmark;
                const uint4 e = cur[j];
                if (!__any_sync(0xFFFFFFFFu, fresh)) {   // the warp's records here were validated before
                    if (in && e.z == lb) pb |= 1u << j;
                    isx[j] = false;
                    same[j] = false;
                    continue;
                }
                const uint32_t u = e.x, vo = e.y, blk = e.z, w3 = e.w;
                const uint32_t tt = w3 & 0xFFFFu, ep = (w3 >> 16) & 0xFFFu, act = (w3 >> 28) & 3u;
                const uint32_t sp = (w3 >> 30) & 1u, resv = w3 >> 31;
                // the record before, loaded by each lane (a coalesced load of the window shifted by one record,
                // mostly from cache): its visit order (strictly increasing) and, in the same block, its epoch
                const uint4 pr = (fresh && idx > 0) ? ev[idx - 1] : make_uint4(0, 0, 0xFFFFFFFFu, 0);
                same[j] = HOT && lane > 0 && pr.z == blk && pr.x == u;
                bool ok = fresh & (blk < nb) & (tt < bt) & (act != 3u) & (resv == 0u) & (u < (sp ? gu : su)) &
                          (idx == 0 || vo > pr.y);
                if (ok && (blk != lb || ep > bmin) && ep > cnts[blk * bt + tt]) ok = false;
                const bool bad = fresh && (!ok || blk != lb);
                const bool back = ok && pr.z == blk && ((pr.w >> 16) & 0xFFFu) > ep;   // epochs go back
                if (__any_sync(0xFFFFFFFFu, bad || back)) {   // rare: a bad record, another block's, epochs going back
                    if (fresh && !ok) atomicMax(&ts[t].bad_rec, ~(unsigned long long)idx);
                    if (ok && blk != lb) atomicOr(&ts[t].inel, 1u);   // the trace is not block-contiguous
                    if (bad || back) stopme = true;
                }
                if (in && blk == lb && (ok || !fresh)) pb |= 1u << j;
                isx[j] = ok && sp == 1u && ep <= maxb;
            }
            uint32_t bal[P], tot = 0;
#pragma unroll
            for (int j = 0; j < P; j++) {
                bal[j] = __ballot_sync(0xFFFFFFFFu, isx[j]);
                tot += __popc(bal[j]);
            }
            if (tot) {
                if (xpos + tot > xend) {   // warp-uniform: a fresh chunk of slots for this warp
                    hb_x_fill(xk, xv, xpos, xend, xcap, lane);
                    uint32_t nbase = 0;
                    if (lane == 0) nbase = atomicAdd(&ctl->n_x, (uint32_t)HB_XCH);
                    nbase = __shfl_sync(0xFFFFFFFFu, nbase, 0);
                    xpos = nbase;
                    xend = nbase + HB_XCH;
                }
                uint32_t before = 0;   // this warp's X records of the items before item j
#pragma unroll
                for (int j = 0; j < P; j++) {
                    const uint32_t bj = bal[j];
                    const uint32_t o = xpos + before + __popc(bj & lt);
                    before += __popc(bj);
                    if (!isx[j]) continue;
                    const uint4 e = cur[j];
                    const uint32_t blk = e.z, w3 = e.w, act = (w3 >> 28) & 3u;
                    const uint32_t xo = pad ? ((blk << 10) | (w3 & 0x3FFu)) : blk * bt + (w3 & 0xFFFFu);
                    if (o < xcap) {
                        xk[o] = (KX)(shl(t, L.bug + L.bxr) | e.x);
                        xv[o] = make_payload(act, xo, e.y);
                    }
                    // a unit every thread reads (a kernel-wide constant) is marked once per run of lanes
                    if (!(same[j] && ((bj >> (lane - 1)) & 1u)))
                        sig_mark(L, sig_t, sig_slot(L, 0ull, t, e.x), blk, d.block_off + blk);
                }
                xpos += tot;
            }
            if (stopme) S.flag = 1u;
            vmark = max(vmark, min(wbase + (uint32_t)SH::window, s1));
            return pb;
        };
        load(cur, s0);
        uint32_t pend = activate();

        uint32_t e = (ev[s0].w >> 16) & 0xFFFu;   // epoch of the block's first record
        uint32_t prev_e = HB_NONE, par = 0, cnt_prev = 0, run_start = s0;
        bool hashing = true, full_reset = false;
        for (;;) {
            uint32_t *kt = key + par * SH::gslots;
            uint64_t *ot = own + par * SH::gslots;
            const uint32_t *pkt = key + (par ^ 1u) * SH::gslots;   // the previous run's table
            const uint64_t *pot = own + (par ^ 1u) * SH::gslots;
            const bool adj = prev_e != HB_NONE && prev_e + 1 == e;
            volatile uint32_t *needed_flag = &S.needed[par];
            // ---- 1. insert run e: its records in this window and, while it goes on, the next windows.
            //      Adjacency (barrier e-1 needed) is tested record by record against the previous run's
            //      table: a conflict between epoch e-1 and the epoch-e records exists exactly when one
            //      record conflicts with it; the test stops once some thread has found one.
            for (;;) {
                const uint32_t wend = min(wbase + (uint32_t)SH::window, s1);
                bool more = false;   // the run goes on past this window: fetch the next one now
                if (wend < s1) {
                    const uint4 last = ev[wend - 1];
                    more = last.z == lb && ((last.w >> 16) & 0xFFFu) == e;
                }
                if (more) load(nxt, wend);
                uint32_t first = HB_NONE;   // the window's first record after the run
#pragma unroll
                for (int j = 0; j < P; j++) {
                    const uint4 r = cur[j];
                    const uint32_t idx = wbase + j * SH::gthreads + tid;
                    const uint32_t ep = (r.w >> 16) & 0xFFFu;
                    const bool mine = ((pend >> j) & 1u) && ep == e;
                    uint32_t s = HB_EMPTY;
                    bool created = false;
                    if (mine) {
                        const uint32_t k = (r.x << 1) | ((r.w >> 30) & 1u);
                        uint32_t h = hb_hash<SH>(k);
                        // linear probing; each probe is a claim attempt (most records bring a new unit,
                        // so the compare-and-swap replaces a plain read rather than following one)
                        for (int probe = 0; probe < SH::gslots; probe++) {
                            const uint32_t old = atomicCAS(&kt[h], HB_EMPTY, k);
                            if (old == HB_EMPTY) { s = h; created = true; break; }
                            if (old == k) { s = h; break; }
                            h = (h + 1) & (SH::gslots - 1);
                        }
                        const uint64_t qb = hb_own_bits((r.w >> 28) & 3u, r.w & 0x3FFu);
                        if (s == HB_EMPTY) {
                            S.flag = 2u;   // table full
                        } else {
                            atomicOr(reinterpret_cast<unsigned long long *>(&ot[s]), (unsigned long long)qb);
                        }
                        if (adj && !*needed_flag) {
                            uint32_t ph = hb_hash<SH>(k);
                            for (int probe = 0; probe < SH::gslots; probe++) {
                                const uint32_t c = pkt[ph];
                                if (c == HB_EMPTY) break;
                                if (c == k) {
                                    if (hb_cross(pot[ph], qb)) *needed_flag = 1u;
                                    break;
                                }
                                ph = (ph + 1) & (SH::gslots - 1);
                            }
                        }
                    } else if (idx < s1) {
                        first = min(first, idx);
                    }
                    const uint32_t cm = __ballot_sync(0xFFFFFFFFu, created);
                    if (cm) {
                        const int leader = __ffs(cm) - 1;
                        uint32_t base = 0;
                        if (lane == leader) base = atomicAdd(&S.cnt[par], (uint32_t)__popc(cm));
                        base = __shfl_sync(0xFFFFFFFFu, base, leader);
                        if (created) {
                            const uint32_t pos = base + __popc(cm & lt);
                            if (pos < cap_rt) list[par * SH::cap + pos] = (uint16_t)s;
                            else S.flag = 2u;   // more distinct units than listed entries
                        }
                    }
                }
                first = __reduce_min_sync(0xFFFFFFFFu, first);
                if (lane == 0 && first != HB_NONE) atomicMin(&S.first[par], first);
                if (more) {
                    wbase = wend;
#pragma unroll
                    for (int j = 0; j < P; j++) cur[j] = nxt[j];
                    pend = activate();
                    continue;
                }
                break;
            }

            // ---- 2. finalise run e
            hb_sync<SH>();   // A: the run's inserts are complete
            const uint32_t flag = S.flag, first = S.first[par];
            const uint32_t cnt = min(S.cnt[par], (uint32_t)SH::cap);
            const uint32_t lo = run_start, hi = (first != HB_NONE ? first : min(wbase + (uint32_t)SH::window, s1)) - 1;
            const uint32_t next_start = hi + 1;
            const bool stop = flag != 0u;
            // the next run's first window: fetched now, it arrives while this run is finalised
            uint32_t next_e = HB_NONE;
            if (!stop && next_start < s1) {
                load(cur, next_start);
                next_e = (ev[next_start].w >> 16) & 0xFFFu;
            }
            if (!stop && tid == 0 && *needed_flag) mark_needed(nonred, L, b, e - 1);
            uint32_t rmask = 0;   // bit m: this thread's list entry tid + m * SH::gthreads is racy
            if (!stop) {
#pragma unroll 1
                for (uint32_t i = tid, m = 0; i < cnt; i += SH::gthreads, m++) {
                    if (hb_racy(ot[list[par * SH::cap + i]])) {
                        rmask |= 1u << m;
                        atomicAdd(&S.nracy[par], 1u);
                    }
                }
                // the previous run's table is no longer read: release it for the next run
                const uint32_t pp = par ^ 1u;
                for (uint32_t i = tid; i < cnt_prev; i += SH::gthreads) {
                    const uint32_t sl = list[pp * SH::cap + i];
                    key[pp * SH::gslots + sl] = HB_EMPTY;
                    own[pp * SH::gslots + sl] = 0ull;
                }
            }
            if (tid == 0) {   // the next run's scalars
                S.cnt[par ^ 1u] = 0;
                S.first[par ^ 1u] = HB_NONE;
                S.nracy[par ^ 1u] = 0;
                S.needed[par ^ 1u] = 0;
            }
            hb_sync<SH>();   // B
            const uint32_t nracy = S.nracy[par];
            if (!stop && nracy > 0) {
                if (nracy > pool_rt || hi - lo >= HB_POS_LIMIT) {
                    // too many racy units: the sort path computes this run's races
                    if (tid == 0) {
                        atomicOr(&spill[(uint64_t)b * L.swords + (e >> 5)], 1u << (e & 31));
                        for (uint32_t tl = lo / IN_TILE; tl <= hi / IN_TILE; tl++) tflag[d.tile_off + tl] = 1u;
                    }
                } else {
                    // exact lowest pairs of the racy units: per category the first item, then the first
                    // item of another thread. The previous run's table was released before barrier B, so
                    // its keys are all HB_EMPTY (every 16-bit half 0xFFFF) and its owner summaries all 0:
                    // the keys become a map slot -> racy index, the summaries the pool of 6 items per
                    // racy unit, and only what the racy units used is put back afterwards.
                    uint16_t *rmap = reinterpret_cast<uint16_t *>(key + (par ^ 1u) * SH::gslots);
                    uint32_t *pool = reinterpret_cast<uint32_t *>(own + (par ^ 1u) * SH::gslots);
                    for (uint32_t i = tid; i < nracy * 6; i += SH::gthreads) pool[i] = HB_EMPTY;
                    for (uint32_t m = 0; rmask >> m; m++)
                        if ((rmask >> m) & 1u)
                            rmap[list[par * SH::cap + tid + m * SH::gthreads]] = (uint16_t)atomicAdd(&S.ridx, 1u);
                    hb_sync<SH>();
                    // a record of a racy unit of this run: racy index | category << 16 in the high word,
                    // run position << 10 | tid in the low word; ~0 for any other record
                    auto racy_item = [&](const uint4 &r, uint32_t i) -> uint64_t {
                        if (r.z != lb || ((r.w >> 16) & 0xFFFu) != e) return ~0ull;
                        const uint32_t c = (r.w >> 28) & 3u;
                        if (c == 3u) return ~0ull;
                        const uint32_t k = (r.x << 1) | ((r.w >> 30) & 1u);
                        uint32_t h = hb_hash<SH>(k);
                        bool found = false;
                        for (int probe = 0; probe < SH::gslots; probe++) {
                            const uint32_t kk = kt[h];
                            if (kk == k) { found = true; break; }
                            if (kk == HB_EMPTY) break;
                            h = (h + 1) & (SH::gslots - 1);
                        }
                        if (!found) return ~0ull;
                        const uint32_t ri = rmap[h];
                        if (ri == 0xFFFFu) return ~0ull;
                        return ((uint64_t)(ri | (c << 16)) << 32) | (((i - lo) << 10) | (r.w & 0x3FFu));
                    };
                    auto first_pass = [&](uint64_t x) {
                        if (x == ~0ull) return;
                        const uint32_t hw = (uint32_t)(x >> 32);
                        atomicMin(&pool[(hw & 0xFFFFu) * 6 + (hw >> 16)], (uint32_t)x);
                    };
                    auto second_pass = [&](uint64_t x) {
                        if (x == ~0ull) return;
                        const uint32_t hw = (uint32_t)(x >> 32), item = (uint32_t)x;
                        uint32_t *pe = pool + (hw & 0xFFFFu) * 6;
                        if ((pe[hw >> 16] & 0x3FFu) != (item & 0x3FFu)) atomicMin(&pe[3 + (hw >> 16)], item);
                    };
                    const uint32_t nrec = hi - lo + 1;
                    if (nrec <= (uint32_t)(SH::gthreads * HB_RM)) {
                        // the run's records, HB_RM per thread, looked up once: both passes use the items
                        uint4 rr[HB_RM];
#pragma unroll
                        for (int m = 0; m < HB_RM; m++) {
                            const uint32_t i = lo + tid + m * SH::gthreads;
                            rr[m] = i <= hi ? ev[i] : make_uint4(0, 0, 0xFFFFFFFFu, 0);
                        }
                        uint64_t it[HB_RM];
#pragma unroll
                        for (int m = 0; m < HB_RM; m++) {
                            it[m] = racy_item(rr[m], lo + tid + m * SH::gthreads);
                            first_pass(it[m]);
                        }
                        hb_sync<SH>();
#pragma unroll
                        for (int m = 0; m < HB_RM; m++) second_pass(it[m]);
                        hb_sync<SH>();
                    } else {
#pragma unroll 1
                        for (int pass = 0; pass < 2; pass++) {
                            for (uint32_t i = lo + tid; i <= hi; i += SH::gthreads) {
                                const uint64_t x = racy_item(ev[i], i);
                                if (pass == 0) first_pass(x);
                                else second_pass(x);
                            }
                            hb_sync<SH>();
                        }
                    }
                    // emission; each racy unit's map entry and pool items are read by its own thread only,
                    // which then puts them back (map entry HB_EMPTY's half, items 0)
                    const OwnThread ownt;
                    for (uint32_t m = 0; rmask >> m; m++) {
                        if (!((rmask >> m) & 1u)) continue;
                        const uint32_t sl = list[par * SH::cap + tid + m * SH::gthreads];
                        const uint32_t k = kt[sl];
                        uint32_t *pe = pool + rmap[sl] * 6;
                        Top2 S;
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            S.a[c] = hb_item64(pe[c]);
                            S.b[c] = hb_item64(pe[3 + c]);
                        }
                        rmap[sl] = 0xFFFFu;
#pragma unroll
                        for (int c = 0; c < 6; c++) pe[c] = 0u;
#pragma unroll
                        for (int cls = 0; cls < 2; cls++) {
                            uint64_t p, q2;
                            if (!lowest_pair(S, cls, ownt, p, q2)) continue;
                            const uint32_t vp = ev[lo + item_pos(p)].y, vq = ev[lo + item_pos(q2)].y;
                            const uint64_t pi = ((uint64_t)vp << 32) | (lb * bt + item_gtid(p));
                            const uint64_t qi = ((uint64_t)vq << 32) | (lb * bt + item_gtid(q2));
                            emit_race(rs, ctl, t, race_key(L, t, k & 1u, 0u, b, e, k >> 1, cls), pi, qi, true);
                        }
                    }
                    if (tid == 0) S.ridx = 0;
                    hb_sync<SH>();   // the map and the pool are clean again before the next run inserts there
                }
            }
            if (stop) {
                // the block goes to the sort path; its tables are cleared in full below
                if (tid == 0) atomicOr(&binel[b], 1u);
                hashing = false;
                full_reset = true;
                break;
            }
            prev_e = e;
            cnt_prev = cnt;
            par ^= 1u;
            run_start = next_start;
            if (next_start >= s1) break;   // the block's last run
            wbase = next_start;
            pend = activate();
            e = next_e;
        }
        // records of the range not yet read (the block left the hash path early): validate and route
        while (vmark < s1) {
            wbase = vmark;
            load(cur, wbase);
            activate();
        }
        // clean tables for the next block
        if (full_reset) {
            hb_sync<SH>();
            for (int i = tid; i < 2 * SH::gslots; i += SH::gthreads) {
                own[i] = 0ull;
                key[i] = HB_EMPTY;
            }
            if (tid == 0) S.flag = 0;
        } else if (hashing) {
            const uint32_t pp = par ^ 1u;   // the last run's table
            for (uint32_t i = tid; i < cnt_prev; i += SH::gthreads) {
                const uint32_t sl = list[pp * SH::cap + i];
                key[pp * SH::gslots + sl] = HB_EMPTY;
                own[pp * SH::gslots + sl] = 0ull;
            }
        }
        if (tid == 0)
            for (int q = 0; q < 2; q++) {
                S.cnt[q] = 0;
                S.first[q] = HB_NONE;
                S.nracy[q] = 0;
                S.needed[q] = 0;
            }
    }
    hb_x_fill(xk, xv, xpos, xend, xcap, lane);   // the unused tail of this warp's last chunk
}

}  // namespace simk
