// fitness.cuh - the fitness of Eq. 1 (Sec. 3.3.1) for a batch of traces.
//
// For memory address i, f(i) is the number of distinct threads that access it
// and g(i) = 1 when it is accessed; F = sum g / sum f (1: no two threads share
// an address; smaller: more sharing, more chances of a conflict). An address
// is a global unit or a shared unit of one block; a thread is its global id;
// every epoch and action counts. The secondary fitness R = end - start uses
// the accessed unit range, reported per space.
//
// Both sums are distinct counts. A distinct (address, thread) pair is a
// distinct (space, unit, thread) triple of one block (thread ids of different
// blocks differ), a distinct shared address is a distinct unit of one block,
// and a distinct global address is a distinct unit of the trace. So one read
// of each block's records does it (k_fit_blocks): one CTA per block inserts the
// block's triples, and the shared units of new triples, into a hash table of
// its own (in global memory, small enough for all CTAs' tables to stay in L2),
// and marks the global units of new triples in a bitmap of the trace's global
// units. New entries and newly set bits are the counts.
//
// What that read cannot do goes to sorting: a block whose entries would fill
// more than 3/4 of the table, and every record of a trace whose blocks are not
// contiguous in record order. Such records become the key (trace | space |
// block for shared | unit | gtid), the keys are radix sorted (keys only), and
// the heads of equal keys count the distinct pairs while the heads of equal
// keys without the gtid field count the distinct addresses (for a block that
// left the table only its shared addresses: its global units are in the
// bitmap, which every global record of the trace marks). Validation is the
// check's (barrier counts, then every record), so a bad trace reports the
// same first bad index.
#pragma once
#include "check_kernels.cuh"
#include "hash_path.cuh"

namespace simk {

struct FitAcc {
    unsigned long long n_addr, n_pairs;   // from the sorted keys
    unsigned long long h_addr, h_pairs;   // from the block tables and the global bitmap
    unsigned int lo[2], hi[2];   // accessed unit range per space (lo > hi: none)
    unsigned int whole;          // every record of the trace is counted from sorted keys
};

// key fields, low to high: gtid (bg) | unit (bu) | block for shared records (bbl) | space (1) | trace (btr)
struct FitKeys {
    uint32_t bg, bu, bbl, btr, bits, np;
};

constexpr int FK_THREADS = 256;
constexpr uint32_t FIT_OUT_BYTES = 48;   // sizeof(simulee_fitness)
constexpr int FK_ITEMS = IN_TILE / FK_THREADS;   // tiles never span traces

__global__ void k_fit_init(const TraceDesc *__restrict__ td, FitAcc *acc, uint32_t T) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        acc[t].n_addr = 0;
        acc[t].n_pairs = 0;
        acc[t].h_addr = 0;
        acc[t].h_pairs = 0;
        acc[t].lo[0] = acc[t].lo[1] = 0xFFFFFFFFu;
        acc[t].hi[0] = acc[t].hi[1] = 0;
        acc[t].whole = td[t].hash_ok ? 0u : 1u;
    }
}

// ---------------------------------------------------------------------------
// The single read: block tables and the global-unit bitmap
// ---------------------------------------------------------------------------
constexpr int FB_THREADS = 1024;
constexpr uint32_t FB_LOG_SLOTS = 16;
constexpr uint32_t FB_SLOTS = 1u << FB_LOG_SLOTS;  // table entries of a CTA (8 bytes each: 512 KB)
constexpr unsigned long long FB_EMPTY = ~0ull;
// A block uses the first 2^lg entries, the smallest power of two (at least 1024) above three times its
// records (it makes at most two entries per record), so a block of few records clears and probes a small
// table; it may fill 3/4 of them before its pairs go to the sort.

// table key: address entry (1 bit) | space (1) | unit (31) | thread (10)
__device__ __forceinline__ unsigned long long fb_key(uint32_t addr, uint32_t sp, uint32_t unit, uint32_t tid) {
    return ((unsigned long long)addr << 42) | ((unsigned long long)sp << 41) |
           ((unsigned long long)(unit & 0x7FFFFFFFu) << 10) | (tid & 0x3FFu);
}

__device__ __forceinline__ uint32_t fb_hash(unsigned long long k, uint32_t lg) {
    return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> (64u - lg));   // Fibonacci hashing, top lg bits
}

// insert k into a table of 2^lg entries, probing from slot h on: 1 new, 0 present, -1 no free slot
__device__ __forceinline__ int fb_insert_from(unsigned long long *tab, unsigned long long k, uint32_t lg, uint32_t h,
                                              uint32_t probes) {
    const uint32_t mask = (1u << lg) - 1u;
    for (uint32_t p = 0; p < probes; p++) {
        const unsigned long long old = atomicCAS(&tab[h], FB_EMPTY, k);
        if (old == FB_EMPTY) return 1;
        if (old == k) return 0;
        h = (h + 1) & mask;
    }
    return -1;
}

// the result of a first claim attempt `old` at k's home slot, probing on when another key holds it
__device__ __forceinline__ int fb_resolve(unsigned long long *tab, unsigned long long k, uint32_t lg,
                                          unsigned long long old) {
    if (old == FB_EMPTY) return 1;
    if (old == k) return 0;
    return fb_insert_from(tab, k, lg, (fb_hash(k, lg) + 1) & ((1u << lg) - 1u), (1u << lg) - 1u);
}

// first record of every block (blocks of traces that take the single read)
__global__ void k_fit_ranges(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, Layout L,
                             uint32_t *bstart) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = warp; b < L.NB; b += nwarps) {
        const TraceDesc &d = td[tob[b]];
        if (!d.hash_ok) continue;
        const uint64_t lo = hb_lower_bound(d, (uint32_t)(b - d.block_off), lane);
        if (lane == 0) bstart[b] = (uint32_t)lo;
    }
}

// One CTA per block, taken from a queue: the block's distinct triples and shared units in the CTA's
// table (cleared for each block), the trace's global units in the bitmap gbits (the trace's units start
// at bit d.sig_off). A record of another block inside the block's range: the trace is counted from
// sorted keys (acc.whole). More than 3/4 of its table's entries: the block's pairs and shared units are counted from
// sorted keys (fb[b]), while its remaining global records still mark the bitmap.
__global__ void __launch_bounds__(FB_THREADS, 1)
k_fit_blocks(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, const uint32_t *__restrict__ bstart,
             Layout L, const TState *ts, unsigned int *queue, unsigned long long *tabs, uint32_t *gbits, FitAcc *acc,
             uint32_t *fb) {
    __shared__ uint32_t s_blk, s_ins, s_over;
    __shared__ unsigned long long s_pairs, s_addr, s_gaddr;
    __shared__ uint32_t s_lo[2], s_hi[2];
    const int tid = threadIdx.x, lane = tid & 31;
    unsigned long long *tab = tabs + (uint64_t)blockIdx.x * FB_SLOTS;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_blk = atomicAdd(queue, 1u);
            s_ins = 0;
            s_over = 0;
            s_pairs = s_addr = s_gaddr = 0;
            s_lo[0] = s_lo[1] = 0xFFFFFFFFu;
            s_hi[0] = s_hi[1] = 0;
        }
        __syncthreads();
        if (s_blk >= L.NB) break;
        const uint32_t b = s_blk, t = tob[b];
        const TraceDesc &d = td[t];
        const volatile TState *v = &ts[t];
        if (!d.hash_ok || v->bad_cnt || v->bad_rec || *(volatile unsigned int *)&acc[t].whole) continue;
        const uint32_t lb = b - d.block_off;
        const uint32_t s0 = bstart[b], s1 = lb + 1 < d.nb ? bstart[b + 1] : (uint32_t)d.n;
        if (s0 >= s1) continue;
        uint32_t lg = 10;
        while (lg < FB_LOG_SLOTS && (1ull << lg) < 3ull * (s1 - s0)) lg++;
        const uint32_t cap = (1u << lg) / 4 * 3;
        // a clean table for this block (the previous block's entries are of no use)
        for (uint32_t i = tid; i < (1u << lg) / 2; i += FB_THREADS)
            reinterpret_cast<ulonglong2 *>(tab)[i] = make_ulonglong2(FB_EMPTY, FB_EMPTY);
        __syncthreads();
        uint32_t lo0 = 0xFFFFFFFFu, hi0 = 0, lo1 = 0xFFFFFFFFu, hi1 = 0;
        uint32_t pairs = 0, addrs = 0, gaddrs = 0;
        // four records per thread per round, their first claim attempts (then the shared units' and the
        // bitmap's atomics) in flight together: the table lives in L2, so each atomic waits out an L2 round
        // trip (two records per round, one after the other: 7% slower)
        constexpr int FR = 4;
        for (uint32_t base = s0; base < s1; base += FR * FB_THREADS) {
            const bool over = *(volatile uint32_t *)&s_over != 0u;
            uint4 e[FR];
#pragma unroll
            for (int j = 0; j < FR; j++) {
                const uint32_t i = base + j * FB_THREADS + tid;
                e[j] = i < s1 ? __ldcs(&d.events[i]) : make_uint4(0, 0, 0xFFFFFFFFu, 0);
            }
            uint32_t live = 0;   // bit j: record j is this block's and in range
#pragma unroll
            for (int j = 0; j < FR; j++) {
                const uint32_t i = base + j * FB_THREADS + tid;
                if (i >= s1) continue;
                if (e[j].z != lb) {   // the trace's blocks are not contiguous: count it from sorted keys
                    atomicOr(&acc[t].whole, 1u);
                    continue;
                }
                live |= 1u << j;
                const uint32_t u = e[j].x;
                if ((e[j].w >> 30) & 1u) { lo1 = min(lo1, u); hi1 = max(hi1, u); }
                else { lo0 = min(lo0, u); hi0 = max(hi0, u); }
            }
            uint32_t made = 0, fresh = over ? live : 0u, newsh = 0;
            if (!over) {
                unsigned long long kk[FR], old[FR];
#pragma unroll
                for (int j = 0; j < FR; j++) {
                    kk[j] = fb_key(0u, (e[j].w >> 30) & 1u, e[j].x, e[j].w & 0xFFFFu);
                    old[j] = ((live >> j) & 1u) ? atomicCAS(&tab[fb_hash(kk[j], lg)], FB_EMPTY, kk[j]) : 0ull;
                }
#pragma unroll
                for (int j = 0; j < FR; j++) {
                    if (!((live >> j) & 1u)) continue;
                    const int r = fb_resolve(tab, kk[j], lg, old[j]);
                    if (r < 0) {
                        s_over = 1u;
                        fresh |= 1u << j;
                    } else if (r > 0) {
                        made++;
                        pairs++;
                        fresh |= 1u << j;
                        if (!((e[j].w >> 30) & 1u)) newsh |= 1u << j;
                    }
                }
                // the shared unit of each new shared pair, first claim attempts together
#pragma unroll
                for (int j = 0; j < FR; j++) {
                    kk[j] = fb_key(1u, 0u, e[j].x, 0u);
                    old[j] = ((newsh >> j) & 1u) ? atomicCAS(&tab[fb_hash(kk[j], lg)], FB_EMPTY, kk[j]) : 0ull;
                }
#pragma unroll
                for (int j = 0; j < FR; j++) {
                    if (!((newsh >> j) & 1u)) continue;
                    const int ra = fb_resolve(tab, kk[j], lg, old[j]);
                    if (ra < 0) s_over = 1u;
                    else if (ra > 0) { made++; addrs++; }
                }
            }
            // global units of new pairs (of every global record once the table is given up), together
            uint32_t was[FR], mbit[FR];
#pragma unroll
            for (int j = 0; j < FR; j++) {
                const bool g = ((fresh >> j) & 1u) && ((e[j].w >> 30) & 1u);
                const uint64_t bit = d.sig_off + e[j].x;
                mbit[j] = g ? 1u << (bit & 31u) : 0u;
                was[j] = g ? atomicOr(&gbits[bit >> 5], mbit[j]) : ~0u;
            }
#pragma unroll
            for (int j = 0; j < FR; j++)
                if (mbit[j] && !(was[j] & mbit[j])) gaddrs++;
            made = __reduce_add_sync(0xFFFFFFFFu, made);
            if (lane == 0 && made && atomicAdd(&s_ins, made) + made > cap) s_over = 1u;
        }
        // the block's sums and ranges
        pairs = __reduce_add_sync(0xFFFFFFFFu, pairs);
        addrs = __reduce_add_sync(0xFFFFFFFFu, addrs);
        gaddrs = __reduce_add_sync(0xFFFFFFFFu, gaddrs);
        lo0 = __reduce_min_sync(0xFFFFFFFFu, lo0);
        hi0 = __reduce_max_sync(0xFFFFFFFFu, hi0);
        lo1 = __reduce_min_sync(0xFFFFFFFFu, lo1);
        hi1 = __reduce_max_sync(0xFFFFFFFFu, hi1);
        if (lane == 0) {
            if (pairs) atomicAdd(&s_pairs, (unsigned long long)pairs);
            if (addrs) atomicAdd(&s_addr, (unsigned long long)addrs);
            if (gaddrs) atomicAdd(&s_gaddr, (unsigned long long)gaddrs);
            if (lo0 <= hi0) { atomicMin(&s_lo[0], lo0); atomicMax(&s_hi[0], hi0); }
            if (lo1 <= hi1) { atomicMin(&s_lo[1], lo1); atomicMax(&s_hi[1], hi1); }
        }
        __syncthreads();
        if (tid == 0) {
            if (s_over) {
                fb[b] = 1u;   // its pairs and shared units from sorted keys
            } else {
                if (s_pairs) atomicAdd(&acc[t].h_pairs, s_pairs);
                if (s_addr) atomicAdd(&acc[t].h_addr, s_addr);
            }
            if (s_gaddr) atomicAdd(&acc[t].h_addr, s_gaddr);
            for (int q = 0; q < 2; q++)
                if (s_lo[q] <= s_hi[q]) {
                    atomicMin(&acc[t].lo[q], s_lo[q]);
                    atomicMax(&acc[t].hi[q], s_hi[q]);
                }
        }
    }
}

__device__ __forceinline__ uint64_t fit_key(const FitKeys &f, uint32_t t, uint32_t sp, uint32_t blk, uint32_t unit,
                                            uint32_t gtid) {
    const uint64_t mg = (f.bg >= 64) ? ~0ull : ((1ull << f.bg) - 1), mu = (1ull << f.bu) - 1, mb = (1ull << f.bbl) - 1;
    uint64_t k = (uint64_t)gtid & mg;
    k |= ((uint64_t)unit & mu) << f.bg;
    k |= (sp ? 0ull : ((uint64_t)blk & mb)) << (f.bg + f.bu);
    k |= (uint64_t)sp << (f.bg + f.bu + f.bbl);
    k |= shl(t, f.bg + f.bu + f.bbl + 1);
    return k;
}

// keys of the records counted from sorted keys (every record of a trace with acc.whole, the records of
// blocks with fb set), compacted (ctl->n_q counts them); their digit histograms; the per-space unit
// ranges of whole traces. One tile (2048 records of one trace) at a time.
template <class K>
__global__ void __launch_bounds__(FK_THREADS)
k_fit_keys(const TraceDesc *__restrict__ td, Layout L, FitKeys fk, const uint32_t *__restrict__ fb, K *keys,
           uint32_t *hist, FitAcc *acc, Ctl *ctl) {
    __shared__ uint32_t sh[8 * RADIX];
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < 8 * RADIX; i += FK_THREADS) sh[i] = 0;
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < L.ntiles_in; tile += gridDim.x) {
        const uint32_t t = trace_of_tile(td, L.T, tile);
        const TraceDesc &d = td[t];
        const bool whole = *(volatile unsigned int *)&acc[t].whole != 0u;
        const uint64_t tbase = (tile - d.tile_off) * IN_TILE;
        uint32_t lo[2] = {0xFFFFFFFFu, 0xFFFFFFFFu}, hi[2] = {0, 0};
#pragma unroll 4
        for (int j = 0; j < FK_ITEMS; j++) {
            const uint64_t idx = tbase + j * FK_THREADS + tid;
            const bool in = idx < d.n;
            const uint4 e = in ? d.events[idx] : make_uint4(0, 0, 0, 0);
            const uint32_t sp = (e.w >> 30) & 1u, tt = e.w & 0xFFFFu;
            // a validated record's block is below the trace's block count
            const bool emit = in && (whole || fb[(uint64_t)d.block_off + min(e.z, d.nb - 1)] != 0u);
            const uint64_t k = fit_key(fk, t, sp, e.z, e.x, e.z * d.bt + tt);
            const uint32_t em = __ballot_sync(0xFFFFFFFFu, emit);
            if (em) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&ctl->n_q, (uint32_t)__popc(em));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (emit) keys[base + __popc(em & lt)] = (K)k;
            }
            if (in && whole) {
                lo[sp] = min(lo[sp], e.x);
                hi[sp] = max(hi[sp], e.x);
            }
            hist_add(sh, k, fk.np, emit, em);
        }
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const uint32_t l = __reduce_min_sync(0xFFFFFFFFu, lo[s]), h = __reduce_max_sync(0xFFFFFFFFu, hi[s]);
            if (lane == 0 && l <= h) {
                atomicMin(&acc[t].lo[s], l);
                atomicMax(&acc[t].hi[s], h);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < (int)(fk.np * RADIX); i += FK_THREADS)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// heads of equal keys in the sorted array: distinct (address, thread) pairs and distinct addresses per trace
template <class K>
__global__ void k_fit_count(const K *__restrict__ keys, const uint32_t *n_ptr, FitKeys fk, uint32_t T, FitAcc *acc,
                            Ctl *ctl) {
    if (must_stop(ctl)) return;
    const uint64_t n = *n_ptr;
    const int lane = threadIdx.x & 31;
    const uint32_t tshift = fk.bg + fk.bu + fk.bbl + 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const uint64_t i = base + threadIdx.x;
        uint32_t hp = 0, ha = 0, t = 0;
        if (i < n) {
            const uint64_t k = (uint64_t)keys[i];
            const uint64_t pk = i > 0 ? (uint64_t)keys[i - 1] : 0;
            hp = (i == 0 || pk != k) ? 1u : 0u;
            ha = (i == 0 || (pk >> fk.bg) != (k >> fk.bg)) ? 1u : 0u;
            t = tshift >= 64 ? 0u : (uint32_t)(k >> tshift);
            // a block that left its table counts only its shared addresses here: its global units are in
            // the bitmap, which counts them once for the trace
            if (ha && t < T && ((k >> (fk.bg + fk.bu + fk.bbl)) & 1u) && !*(volatile unsigned int *)&acc[t].whole)
                ha = 0;
        }
        const uint32_t active = __ballot_sync(0xFFFFFFFFu, i < n);
        const uint32_t t0 = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (__all_sync(0xFFFFFFFFu, i >= n || t == t0)) {
            const uint32_t sp = __reduce_add_sync(0xFFFFFFFFu, hp), sa = __reduce_add_sync(0xFFFFFFFFu, ha);
            if (lane == 0 && active && t0 < T) {
                if (sp) atomicAdd(&acc[t0].n_pairs, (unsigned long long)sp);
                if (sa) atomicAdd(&acc[t0].n_addr, (unsigned long long)sa);
            }
        } else if (i < n && t < T) {
            if (hp) atomicAdd(&acc[t].n_pairs, 1ull);
            if (ha) atomicAdd(&acc[t].n_addr, 1ull);
        }
    }
}

// simulee_fitness per trace: status and first bad index (as the check reports them), sums, ranges
__global__ void k_fit_report(const TState *ts, const FitAcc *acc, uint32_t T, Ctl *ctl, uint8_t *out) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const volatile TState *v = &ts[t];
        int32_t status = 0;
        uint32_t kind = 0;
        uint64_t bad = 0, na = acc[t].n_addr, np = acc[t].n_pairs;
        if (!acc[t].whole) {   // the single read's counts, plus those of blocks that left their table
            na += acc[t].h_addr;
            np += acc[t].h_pairs;
        }
        if (v->bad_cnt) {
            status = 2; kind = 1; bad = ~v->bad_cnt;
        } else if (v->bad_rec) {
            status = 2; kind = 0; bad = ~v->bad_rec;
        } else if (*(volatile unsigned int *)&ctl->timeout) {
            status = 5;
        }
        if (status) { na = 0; np = 0; }
        uint8_t *o = out + FIT_OUT_BYTES * (uint64_t)t;
        reinterpret_cast<int32_t *>(o)[0] = status;
        reinterpret_cast<uint32_t *>(o)[1] = kind;
        reinterpret_cast<uint64_t *>(o)[1] = bad;
        reinterpret_cast<uint64_t *>(o)[2] = na;
        reinterpret_cast<uint64_t *>(o)[3] = np;
        uint32_t *r = reinterpret_cast<uint32_t *>(o + 32);
        r[0] = status ? 0xFFFFFFFFu : acc[t].lo[0];
        r[1] = status ? 0u : acc[t].hi[0];
        r[2] = status ? 0xFFFFFFFFu : acc[t].lo[1];
        r[3] = status ? 0u : acc[t].hi[1];
    }
}

}  // namespace simk
