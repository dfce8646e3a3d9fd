// check_kernels.cuh - ingest, segmented reduction and output kernels of the check.
//
// Every kernel works on a batch of traces described by TraceDesc entries; a
// single-trace call is a batch of one. Blocks are numbered batch-wide (trace
// t's block b is block_off[t] + b), keys of the intra-block streams carry that
// batch-wide block, and the inter-block stream's key carries the trace index,
// so groups never mix traces. Outputs are split back per trace at the end.
#pragma once
#include "common.cuh"
#include "sort.cuh"

namespace simk {

__device__ __forceinline__ uint32_t trace_of_tile(const TraceDesc *td, uint32_t T, uint64_t tile) {
    return find_trace(T, tile, [&](uint32_t t) { return td[t].tile_off; });
}

// batch-wide block -> trace
__global__ void k_block_trace(const TraceDesc *td, Layout L, uint32_t *tob) {
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < L.NB; b += (uint64_t)gridDim.x * blockDim.x)
        tob[b] = find_trace(L.T, b, [&](uint32_t t) { return (uint64_t)td[t].block_off; });
}

// ---------------------------------------------------------------------------
// Barrier counts: per-block min / max / first thread at the min (Algorithm 4's
// divergence test is "threads of a block reached different barrier counts"),
// plus validation of every count. One warp per block.
// stats[b] = (min, min(max, max_barriers), first tid at min, max).
// ---------------------------------------------------------------------------
__global__ void k_block_stats(const TraceDesc *td, const uint32_t *tob, Layout L, uint4 *stats, TState *ts) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = warp; b < L.NB; b += nwarps) {
        const uint32_t t = tob[b];
        const TraceDesc &d = td[t];
        const uint64_t lb = b - d.block_off;
        const uint32_t *cnt = d.counts + lb * d.bt;
        uint32_t mn = 0xFFFFFFFFu, mx = 0, first = 0xFFFFFFFFu;
        for (uint32_t i = lane; i < d.bt; i += 32) {
            const uint32_t c = cnt[i];
            if (c > d.maxb) atomicMax(&ts[t].bad_cnt, ~(unsigned long long)(lb * d.bt + i));
            if (c < mn) { mn = c; first = i; }
            mx = max(mx, c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t omn = __shfl_xor_sync(0xFFFFFFFFu, mn, o);
            const uint32_t ofi = __shfl_xor_sync(0xFFFFFFFFu, first, o);
            mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            if (omn < mn || (omn == mn && ofi < first)) { mn = omn; first = ofi; }
        }
        if (lane == 0) stats[b] = make_uint4(mn, min(mx, L.maxb), first, mx);
    }
}

__device__ __forceinline__ uint32_t digit_of(uint64_t k, uint32_t p) { return (uint32_t)(k >> (8 * p)) & (RADIX - 1); }

// x << s for s in [0, 64], defined for s == 64
__device__ __forceinline__ uint64_t shl(uint64_t x, uint32_t s) { return s >= 64 ? 0ull : x << s; }

// Add the digits of every pass of a key to shared histograms; when the whole
// warp's participating lanes share a digit, one lane adds the warp's count.
__device__ __forceinline__ void hist_add(uint32_t *sh, uint64_t key, uint32_t npass, bool part, uint32_t pmask) {
    if (pmask == 0) return;
    const int leader = __ffs(pmask) - 1;
    const int lane = threadIdx.x & 31;
    for (uint32_t p = 0; p < npass; p++) {
        const uint32_t d = part ? digit_of(key, p) : 0u;
        const uint32_t dl = __shfl_sync(0xFFFFFFFFu, d, leader);
        const bool uni = __all_sync(0xFFFFFFFFu, !part || d == dl);
        if (uni) {
            if (lane == leader) atomicAdd(&sh[p * RADIX + d], (uint32_t)__popc(pmask));
        } else if (part) {
            atomicAdd(&sh[p * RADIX + d], 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// Block signatures of global units. An inter-block race needs a unit touched
// by two different blocks. Each global record marks its unit's slot; records
// whose slot shows a single block are dropped before the inter-block sort.
// When every trace has at most 2^15 blocks the slot is the OR of
// (b | ~b << 15) over the trace-local blocks b that touched it: it shows two
// or more blocks exactly when its two 15-bit halves share a bit, and a mark is
// one atomicOr whose result nobody waits for. Otherwise the slot holds the
// batch-wide block + 1, and SIG_MULTI once another block touches it.
// With several traces the slot is a hash of (trace, unit); a collision can
// only keep extra records, never drop a needed one.
// ---------------------------------------------------------------------------
constexpr uint32_t SIG_MULTI = 0x80000000u;

__device__ __forceinline__ uint64_t sig_slot(const Layout &L, uint64_t sig_off, uint32_t t, uint32_t unit) {
    if (L.sig_direct) return sig_off + unit;
    return (mix32((t * 0x9E3779B1u) ^ unit) ^ ((uint64_t)t << 7)) & (L.sig_slots - 1);
}

__device__ __forceinline__ void sig_mark(const Layout &L, uint32_t *sig, uint64_t slot, uint32_t local_block,
                                         uint32_t block) {
    if (L.sig_or) {
        atomicOr(&sig[slot], (local_block & 0x7FFFu) | ((~local_block & 0x7FFFu) << 15));
        return;
    }
    const uint32_t me = block + 1u;
    uint32_t cur = *(volatile uint32_t *)&sig[slot];
    if (cur == me || (cur & SIG_MULTI)) return;
    if (cur == 0u) cur = atomicCAS(&sig[slot], 0u, me);
    if (cur != 0u && cur != me && !(cur & SIG_MULTI)) atomicOr(&sig[slot], SIG_MULTI);
}

__device__ __forceinline__ bool sig_multi(const Layout &L, uint32_t v) {
    return L.sig_or ? ((v & (v >> 15) & 0x7FFFu) != 0u) : (v & SIG_MULTI) != 0u;
}

// ---------------------------------------------------------------------------
// Ingest, in up to two reads of the records.
//
// First read (IN_FIRST), for traces on the sort path: validate every record;
// route global records to the inter-block stream X keyed (trace, unit), shared
// records to stream S and global records to stream G, both keyed (block, unit,
// epoch). Digit histograms of the radix passes are built on the way. Tiles of
// hash-path traces are skipped: the hash path reads those records itself.
// Fallback read (IN_FALLBACK): route S and G for what the hash path left to
// the sort path: every record of a block it gave up on, of a trace whose
// blocks are out of order, and of a spilled (block, epoch) run. It visits only
// the tiles k_fallback_tiles listed.
// Validate-only read (IN_VALIDATE): validation alone.
//
// Tiles of 2048 records (a tile never spans two traces) are staged into shared
// memory by 1-D bulk copies (TMA) on an mbarrier, double-buffered: the copy of
// the CTA's next-but-one tile is in flight while a tile is processed. Each
// copy brings the record before the tile as well, for the order checks. A
// tile is read twice from shared memory: once to validate and count, once to
// write the routed elements at their stream positions.
// ---------------------------------------------------------------------------
constexpr int IN_THREADS = 512;
constexpr int IN_ITEMS = 4;
constexpr int IN_TILE = IN_THREADS * IN_ITEMS;
constexpr int IN_STAGE = IN_TILE + 1;   // records per stage buffer (one before the tile)
constexpr int IN_MAXP = 24;   // S + G + X passes histogrammed here
constexpr int IN_FIRST = 0, IN_FALLBACK = 1, IN_VALIDATE = 2;

constexpr size_t ingest_smem() { return 2 * (size_t)IN_STAGE * 16; }

template <class KS, class KG, class KX, int MODE>
__global__ void __launch_bounds__(IN_THREADS)
k_ingest(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ rank, Layout L, TState *ts, Ctl *ctl,
         KS *sk, uint64_t *sv, KG *gk, uint64_t *gv, KX *xk, uint64_t *xv, uint32_t *hist,
         const uint32_t *__restrict__ binel, const uint32_t *__restrict__ spill, const uint32_t *__restrict__ tile_list,
         uint32_t *sig, uint64_t wait_ns) {
    extern __shared__ __align__(128) uint4 in_stage[];   // [2][IN_STAGE]
    __shared__ uint64_t bars[2];
    __shared__ uint32_t sh[IN_MAXP * RADIX];
    __shared__ uint32_t wtot[IN_THREADS / 32][3];
    __shared__ uint32_t cbase[3];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t np_s = L.np_s, np_g = L.np_g;
    uint32_t *hs = sh, *hg = sh + np_s * RADIX;
    for (int i = tid; i < IN_MAXP * RADIX; i += IN_THREADS) sh[i] = 0;
    const uint64_t ntiles = (MODE == IN_FALLBACK) ? (uint64_t)*(volatile unsigned int *)&ctl->n_fb : L.ntiles_in;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // thread 0: start the copy of this CTA's k-th tile into stage k & 1
    auto issue = [&](uint64_t k) {
        const uint64_t i = blockIdx.x + k * gridDim.x;
        if (i >= ntiles) return;
        const uint64_t tile = (MODE == IN_FALLBACK) ? tile_list[i] : i;
        const TraceDesc &d = td[trace_of_tile(td, L.T, tile)];
        if (MODE == IN_FIRST && d.hash_ok) {
            mbar_arrive_expect_tx(&bars[k & 1], 0u);   // nothing to copy: complete the phase
            return;
        }
        const uint64_t tbase = (tile - d.tile_off) * IN_TILE;
        const uint64_t first = tbase > 0 ? tbase - 1 : 0, last = min(tbase + IN_TILE, d.n);
        const uint32_t bytes = (uint32_t)((last - first) * 16);
        uint4 *dst = in_stage + (k & 1) * IN_STAGE + (tbase > 0 ? 0 : 1);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[k & 1], bytes);
        bulk_g2s(dst, d.events + first, bytes, &bars[k & 1]);
    };
    if (tid == 0) {
        issue(0);
        issue(1);
    }
    for (uint64_t k = 0;; k++) {
        const uint64_t i = blockIdx.x + k * gridDim.x;
        if (i >= ntiles) break;
        const bool arrived = __syncthreads_and(mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1), wait_ns));
        if (!arrived) {
            // bounded: report, give the copies in flight one more bounded wait, and stop
            if (tid == 0) {
                atomicExch(&ctl->timeout, 1u);
                mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1), wait_ns);
                if (i + gridDim.x < ntiles) mbar_wait(&bars[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), wait_ns);
            }
            return;
        }
        const uint64_t tile = (MODE == IN_FALLBACK) ? tile_list[i] : i;
        const uint32_t t = trace_of_tile(td, L.T, tile);
        const TraceDesc &d = td[t];
        const uint64_t tbase = (tile - d.tile_off) * IN_TILE;
        const uint4 *recs = in_stage + (k & 1) * IN_STAGE + 1;   // recs[-1]: the record before the tile
        const bool hash_tr = d.hash_ok != 0;
        if (!(MODE == IN_FIRST && hash_tr)) {   // uniform: a hash-path tile in the first read is skipped
        const bool trace_fb = MODE == IN_FALLBACK && *(volatile uint32_t *)&ts[t].inel != 0;
        const bool sorted = (d.flags & 1u) == 0;
        const bool route_sg_tile = MODE == IN_FIRST || MODE == IN_FALLBACK;
        uint32_t route = 0;   // bit j: S, bit 8+j: G, bit 16+j: X
        uint32_t cS = 0, cG = 0, cX = 0;
        // pass 1: validate, decide routes, count, run bookkeeping, histograms
#pragma unroll
        for (int j = 0; j < IN_ITEMS; j++) {
            const uint32_t li = j * IN_THREADS + tid;
            const uint64_t idx = tbase + li;   // record index in the trace
            const bool in = idx < d.n;
            const uint4 e = in ? recs[li] : make_uint4(0, 0, 0, 0);
            const uint4 pe = (in && idx > 0) ? recs[(int)li - 1] : make_uint4(0, 0, 0, 0);
            const uint32_t u = e.x, vo = e.y, blk = e.z, w3 = e.w;
            const uint32_t tt = w3 & 0xFFFFu, ep = (w3 >> 16) & 0xFFFu, act = (w3 >> 28) & 3u;
            const uint32_t space = (w3 >> 30) & 1u, resv = w3 >> 31;
            bool ok = in && blk < d.nb && tt < d.bt && act != 3u && resv == 0u && (space ? u < d.gu : u < d.su);
            if (ok && ep > d.counts[blk * d.bt + tt]) ok = false;
            if (in && sorted && idx > 0 && vo <= pe.y) ok = false;
            if (MODE != IN_FALLBACK && in && !ok) atomicMax(&ts[t].bad_rec, ~(unsigned long long)idx);
            // routed records also keep the epoch inside the key's epoch field
            const bool rok = MODE != IN_VALIDATE && ok && ep <= d.maxb;
            bool route_sg = route_sg_tile;
            if (MODE == IN_FALLBACK && !trace_fb) {
                const uint64_t sb = (uint64_t)d.block_off + blk;
                route_sg = rok && (binel[sb] != 0 || ((spill[sb * L.swords + (ep >> 5)] >> (ep & 31)) & 1u));
            }
            const bool isS = rok && route_sg && space == 0u, isG = rok && route_sg && space == 1u;
            // inter-block stream: global records (a trace with the paper's visit-order counters gets its
            // elements from the sorted intra-block stream instead, once the counters are known; its units
            // are marked here all the same)
            const bool markX = MODE == IN_FIRST && rok && space == 1u;
            const bool isX = markX && !(d.flags & TF_PAPER_ORDER);
            const uint32_t bS = __ballot_sync(0xFFFFFFFFu, isS), bG = __ballot_sync(0xFFFFFFFFu, isG);
            const uint32_t bX = __ballot_sync(0xFFFFFFFFu, isX);
            // a unit every thread reads (a kernel-wide constant) is marked once per run of lanes
            const uint32_t bM = __ballot_sync(0xFFFFFFFFu, markX);
            const uint32_t pu = __shfl_up_sync(0xFFFFFFFFu, u, 1), pblk = __shfl_up_sync(0xFFFFFFFFu, blk, 1);
            const bool sameM = lane > 0 && ((bM >> (lane - 1)) & 1u) && pu == u && pblk == blk;
            cS += __popc(bS);
            cG += __popc(bG);
            cX += __popc(bX);
            route |= ((isS ? 1u : 0u) << j) | ((isG ? 1u : 0u) << (8 + j)) | ((isX ? 1u : 0u) << (16 + j));
            if (MODE != IN_VALIDATE) {
                const uint64_t sb = (uint64_t)d.block_off + blk;
                if (bS) hist_add(hs, shl(sb, L.bus + L.be) | shl(u, L.be) | ep, np_s, isS, bS);
                if (bG) hist_add(hg, shl(sb, L.bug + L.be) | shl(u, L.be) | ep, np_g, isG, bG);
                if (markX && !sameM) sig_mark(L, sig, sig_slot(L, d.sig_off, t, u), blk, (uint32_t)sb);
            }
        }
        if (MODE != IN_VALIDATE) {
            if (lane == 0) { wtot[w][0] = cS; wtot[w][1] = cG; wtot[w][2] = cX; }
            __syncthreads();
            if (tid == 0) {
                uint32_t a = 0, b = 0, c = 0;
                for (int q = 0; q < IN_THREADS / 32; q++) {
                    const uint32_t x = wtot[q][0], y = wtot[q][1], z = wtot[q][2];
                    wtot[q][0] = a; wtot[q][1] = b; wtot[q][2] = c;
                    a += x; b += y; c += z;
                }
                cbase[0] = a ? atomicAdd(&ctl->n_s, a) : 0u;
                cbase[1] = b ? atomicAdd(&ctl->n_g, b) : 0u;
                cbase[2] = c ? atomicAdd(&ctl->n_x, c) : 0u;
            }
            __syncthreads();
            // pass 2: write the routed elements
            uint32_t oS = cbase[0] + wtot[w][0], oG = cbase[1] + wtot[w][1], oX = cbase[2] + wtot[w][2];
#pragma unroll
            for (int j = 0; j < IN_ITEMS; j++) {
                const bool isS = (route >> j) & 1u, isG = (route >> (8 + j)) & 1u, isX = (route >> (16 + j)) & 1u;
                const uint32_t bS = __ballot_sync(0xFFFFFFFFu, isS), bG = __ballot_sync(0xFFFFFFFFu, isG);
                const uint32_t bX = __ballot_sync(0xFFFFFFFFu, isX);
                if (isS || isG || isX) {
                    const uint32_t li = j * IN_THREADS + tid;
                    const uint64_t idx = tbase + li;
                    const uint4 e = recs[li];
                    const uint32_t u = e.x, blk = e.z, w3 = e.w;
                    const uint32_t ep = (w3 >> 16) & 0xFFFu, act = (w3 >> 28) & 3u;
                    const uint32_t pos = sorted ? e.y : rank[d.rec_off + idx];
                    // warp-aware traces: intra-block elements carry the record index (for the statement word)
                    const uint32_t ipos = (d.flags & TF_WARP_AWARE) ? (uint32_t)idx : pos;
                    const uint64_t val = make_payload(act, blk * d.bt + (w3 & 0xFFFFu), ipos);
                    const uint64_t sb = (uint64_t)d.block_off + blk;
                    if (isS) {
                        const uint32_t o = oS + __popc(bS & lt);
                        if (o < L.cap_s) {   // beyond the capacity: the call reports ENOMEM
                            sk[o] = (KS)(shl(sb, L.bus + L.be) | shl(u, L.be) | ep);
                            sv[o] = val;
                        }
                    }
                    if (isG) {
                        const uint32_t o = oG + __popc(bG & lt);
                        if (o < L.cap_s) {
                            gk[o] = (KG)(shl(sb, L.bug + L.be) | shl(u, L.be) | ep);
                            gv[o] = val;
                        }
                    }
                    if (isX) {
                        // inter-block payload: owner code block << 10 | tid (a shift gives the block)
                        // when blocks fit 20 bits, else the thread id
                        const uint32_t xo = d.nb <= (1u << 20) ? ((blk << 10) | (w3 & 0x3FFu)) : blk * d.bt + (w3 & 0xFFFFu);
                        const uint32_t o = oX + __popc(bX & lt);
                        if (o < L.x_cap) {
                            xk[o] = (KX)(shl(t, L.bug + L.bxr) | u);
                            xv[o] = make_payload(act, xo, pos);
                        }
                    }
                }
                oS += __popc(bS);
                oG += __popc(bG);
                oX += __popc(bX);
            }
        }
        }
        __syncthreads();   // every thread is done with this stage buffer
        if (tid == 0) issue(k + 2);
    }
    __syncthreads();
    if (MODE == IN_VALIDATE) return;
    const uint32_t tot = (np_s + np_g) * RADIX;   // the inter stream is histogrammed by its filter
    for (uint32_t i = tid; i < tot; i += IN_THREADS) {
        const uint32_t c = sh[i];
        if (c) {
            const uint32_t p = i / RADIX;
            const uint32_t gp = p < np_s ? L.p0_s + p : L.p0_g + (p - np_s);
            atomicAdd(&hist[gp * RADIX + (i % RADIX)], c);
        }
    }
}

// Tiles the fallback read must visit: those of hash-path traces holding a block
// that the hash path gave up on or part of a spilled run (or every tile of a
// trace whose blocks are out of order). One thread per tile; the list order
// does not matter.
__global__ void k_fallback_tiles(const TraceDesc *__restrict__ td, Layout L, const TState *ts,
                                 const uint32_t *__restrict__ binel, const uint32_t *__restrict__ tflag, Ctl *ctl,
                                 uint32_t *list) {
    for (uint64_t tile = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; tile < L.ntiles_in;
         tile += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = trace_of_tile(td, L.T, tile);
        const TraceDesc &d = td[t];
        if (!d.hash_ok) continue;
        bool fb = ts[t].inel != 0 || tflag[tile] != 0;
        if (!fb) {
            // blocks are in record order here: the tile covers blocks first..last
            const uint64_t tbase = (tile - d.tile_off) * IN_TILE, last = min(tbase + IN_TILE, d.n) - 1;
            const uint32_t b0 = min(d.events[tbase].z, d.nb - 1), b1 = min(d.events[last].z, d.nb - 1);
            for (uint32_t b = b0; b <= b1 && !fb; b++) fb = binel[(uint64_t)d.block_off + b] != 0;
        }
        if (fb) list[atomicAdd(&ctl->n_fb, 1u)] = (uint32_t)tile;
    }
}

// Keep the inter-block records whose unit was touched by two or more blocks;
// build the digit histograms of the records kept. The order of kept records
// does not matter (the sort that follows groups them by unit). Slots the hash
// path reserved but did not use carry an invalid action and are dropped.
// A CTA takes tiles of 4096 elements (8 per thread); kept elements are
// compacted with warp ballots and one atomicAdd per tile.
constexpr int XF_THREADS = 512;
constexpr int XF_ITEMS = 8;
constexpr int XF_TILE = XF_THREADS * XF_ITEMS;

// OFFS: a direct signature table of several traces (each trace's units after the previous traces')
template <class KX, bool OFFS>
__global__ void __launch_bounds__(XF_THREADS, sizeof(KX) == 4 ? 3 : 2)
k_x_filter(const KX *__restrict__ xk, const uint64_t *__restrict__ xv, KX *yk, uint64_t *yv, const uint32_t *sig,
           const TraceDesc *__restrict__ td, Layout L, Ctl *ctl, uint32_t *hist) {
    __shared__ uint32_t sh[8 * RADIX];
    // warp counts, then offsets, of a tile; two sets used in turn, so that a tile's set is only
    // rewritten two tiles later, after every warp has passed the next tile's first barrier
    __shared__ uint32_t wtot[2][XF_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < 8 * RADIX; i += XF_THREADS) sh[i] = 0;
    __syncthreads();
    const uint64_t n = min((uint64_t)*(volatile unsigned int *)&ctl->n_x, L.x_cap);
    uint32_t par = 0;
    const uint64_t umask = (L.bug >= 64) ? ~0ull : ((1ull << L.bug) - 1);
    for (uint64_t base = (uint64_t)blockIdx.x * XF_TILE; base < n; base += (uint64_t)gridDim.x * XF_TILE) {
        KX k[XF_ITEMS];
        uint32_t sv[XF_ITEMS];
#pragma unroll
        for (int j = 0; j < XF_ITEMS; j++) {
            const uint64_t i = base + j * XF_THREADS + tid;
            k[j] = i < n ? xk[i] : (KX)0;
        }
#pragma unroll
        for (int j = 0; j < XF_ITEMS; j++) {
            const uint64_t i = base + j * XF_THREADS + tid;
            const uint64_t kk = (uint64_t)k[j];
            const uint32_t t = (uint32_t)(L.bug + L.bxr >= 64 ? 0 : (kk >> (L.bug + L.bxr))), unit = (uint32_t)(kk & umask);
            const uint64_t off = (OFFS && i < n && t < L.T) ? td[t].sig_off : 0ull;
            sv[j] = i < n ? sig[sig_slot(L, off, t, unit)] : 0u;
        }
        uint64_t v[XF_ITEMS];
        uint32_t keep = 0;
#pragma unroll
        for (int j = 0; j < XF_ITEMS; j++) {
            const uint64_t i = base + j * XF_THREADS + tid;
            v[j] = 0;
            if (i < n && sig_multi(L, sv[j])) {
                v[j] = xv[i];
                if (payload_act(v[j]) != 3u) keep |= 1u << j;
            }
        }
        // positions: warp ballots per item, warp totals, one atomicAdd per tile
        uint32_t wcount = 0, bal[XF_ITEMS];
#pragma unroll
        for (int j = 0; j < XF_ITEMS; j++) {
            bal[j] = __ballot_sync(0xFFFFFFFFu, (keep >> j) & 1u);
            wcount += __popc(bal[j]);
        }
        if (lane == 0) wtot[par][w] = wcount;
        __syncthreads();
        if (w == 0) {
            const uint32_t x = lane < XF_THREADS / 32 ? wtot[par][lane] : 0u;
            uint32_t incl = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            uint32_t b0 = 0;
            if (lane == 0 && total) b0 = atomicAdd(&ctl->n_xf, total);
            b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
            if (lane < XF_THREADS / 32) wtot[par][lane] = b0 + incl - x;
        }
        __syncthreads();
        if (keep) {
            uint32_t o = wtot[par][w];
#pragma unroll
            for (int j = 0; j < XF_ITEMS; j++) {
                if ((keep >> j) & 1u) {
                    const uint32_t pos = o + __popc(bal[j] & lt);
                    if (pos < L.cap_x1) {   // beyond the capacity: the call reports ENOMEM
                        yk[pos] = k[j];
                        yv[pos] = v[j];
                    }
                    const uint64_t kk = (uint64_t)k[j];
                    for (uint32_t q = 0; q < L.np_x; q++) atomicAdd(&sh[q * RADIX + digit_of(kk, q)], 1u);
                }
                o += __popc(bal[j]);
            }
        }
        par ^= 1u;
    }
    __syncthreads();
    for (int i = tid; i < (int)(L.np_x * RADIX); i += XF_THREADS)
        if (sh[i]) atomicAdd(&hist[(L.p0_x + i / RADIX) * RADIX + (i % RADIX)], sh[i]);
}

// ---------------------------------------------------------------------------
// Race staging: canonical key + payload (vo_first, vo_second, gtid_first, gtid_second).
// Canonical key bits, low to high: cls(1) unit(bu) epoch(be) block(bb) scope(1)
// space(1) trace(btr); the block field holds the batch-wide block, which orders
// a trace's blocks like its own block numbers.
// ---------------------------------------------------------------------------
struct RaceStage {
    uint64_t *keys;
    uint64_t *idx;
    uint4 *pay;
    uint64_t cap;
    const uint32_t *pos_to_vo;   // unsorted traces: schedule position -> visit order (else NULL)
    uint64_t n_pos;              // entries of pos_to_vo
    TState *ts;
    const TraceDesc *td;
};

__device__ __forceinline__ uint64_t race_key(const Layout &L, uint32_t trace, uint32_t space, uint32_t scope,
                                             uint32_t block, uint32_t epoch, uint32_t unit, uint32_t cls) {
    uint64_t k = cls;
    k |= (uint64_t)unit << 1;
    k |= (uint64_t)epoch << (1 + L.bu);
    k |= (uint64_t)block << (1 + L.bu + L.be);
    k |= (uint64_t)scope << (1 + L.bu + L.be + L.bb);
    k |= (uint64_t)space << (2 + L.bu + L.be + L.bb);
    k |= shl(trace, 3 + L.bu + L.be + L.bb);
    return k;
}

// Staged races carry their payload index; bit 63 marks a race of the hash
// path, which the race filter drops when its block fell back to the sort path.
// Capacity: a group of m >= 2 records yields at most min(2, m - 1) <= 2m/3
// races, and each record lies in one intra-block group of the hash path, one
// of the sort path and one inter-block group, so at most 2n races are staged.
constexpr uint64_t RACE_FROM_HASH = 1ull << 63;

__device__ __forceinline__ void emit_race(const RaceStage &rs, Ctl *ctl, uint32_t trace, uint64_t key, uint64_t p,
                                          uint64_t q, bool from_hash = false) {
    const uint32_t slot = atomicAdd(&ctl->n_races, 1u);
    atomicAdd(&rs.ts[trace].n_races, 1u);
    if (slot < rs.cap) {
        rs.keys[slot] = key;
        rs.idx[slot] = slot | (from_hash ? RACE_FROM_HASH : 0ull);
        uint32_t vp = item_pos(p), vq = item_pos(q);
        if (rs.pos_to_vo && (rs.td[trace].flags & 1u)) {
            vp = vp < rs.n_pos ? rs.pos_to_vo[vp] : 0u;
            vq = vq < rs.n_pos ? rs.pos_to_vo[vq] : 0u;
        }
        rs.pay[slot] = make_uint4(vp, vq, item_gtid(p), item_gtid(q));
    }
}

template <class Own>
__device__ __forceinline__ void emit_group(const Layout &L, const RaceStage &rs, Ctl *ctl, const Top2 &s,
                                           const Own &own, uint32_t trace, uint32_t space, uint32_t scope,
                                           uint32_t block, uint32_t epoch, uint32_t unit) {
#pragma unroll
    for (int cls = 0; cls < 2; cls++) {
        uint64_t p, q;
        if (lowest_pair(s, cls, own, p, q))
            emit_race(rs, ctl, trace, race_key(L, trace, space, scope, block, epoch, unit, cls), p, q);
    }
}

// barrier k of batch-wide block b is needed (not redundant)
__device__ __forceinline__ void mark_needed(uint32_t *nonred, const Layout &L, uint32_t block, uint32_t k) {
    if (block < L.NB && (k >> 5) < L.words) atomicOr(&nonred[(uint64_t)block * L.words + (k >> 5)], 1u << (k & 31));
}

// The same for callers that mark per conflicting group: every conflicting pair of adjacent epochs of
// every unit of a block marks the same word, so the atomic is skipped once the bit is visible (bits only
// go from 0 to 1: a stale read only costs the atomic). Without that the atomics on one word queue up one
// after another: a sorted stream's reduction ran 5x longer.
__device__ __forceinline__ void mark_needed_once(uint32_t *nonred, const Layout &L, uint32_t block, uint32_t k) {
    if (block < L.NB && (k >> 5) < L.words) {
        uint32_t *w = &nonred[(uint64_t)block * L.words + (k >> 5)];
        const uint32_t bit = 1u << (k & 31);
        if (!(*(volatile uint32_t *)w & bit)) atomicOr(w, bit);
    }
}

// ---------------------------------------------------------------------------
// Segmented reductions over a sorted stream: the conflict scan.
//
// CTAs claim tiles of 2048 sorted elements in order. A tile is loaded into
// shared memory and cut at its group heads (key changes) into segments: the
// piece before its first head (the end of a group that began in an earlier
// tile), the groups that begin and end inside it, and its last piece, which
// may run on into later tiles. A segment is reduced to its top-2 summary by
// one thread when it is short and by a warp when it is long: the lanes stride
// over it and their summaries are merged with warp-wide min reductions (all
// the segment's elements are accesses of one unit, so this groups same-unit
// accesses inside a warp).
//
// A group is finished (races emitted, adjacency tested) by the tile that holds
// its last element. Before it waits on anything, every tile publishes the
// summary of its last piece and of the piece before its last head and then a
// ready word tagged with the launch; a group that began in earlier tiles is
// completed by looking back over those summaries until the tile holding its
// head (256 tiles per step). Tiles are claimed in order and publish before they
// wait, so every wait is on a tile already being processed, and waits are
// bounded by wall time as in the radix sort. A group of millions of elements
// is thus summarised by all the tiles it covers at once and finished by one
// look-back over their summaries.
//
// Intra streams (key = block, unit, epoch with the epoch in the low bits):
// group (b, u, e) and the group before it are epochs e-1 and e of the same unit
// exactly when the key before is key - 1 (with the paper's visit-order counters:
// when both have the same block and unit); a conflict between their summaries
// marks barrier e-1 of block b as needed. The finisher of the later group tests
// the pair.
// Inter stream (key = trace, global unit): owners are blocks; no adjacency.
// ---------------------------------------------------------------------------
constexpr int RG_THREADS = 256;
constexpr int RG_ITEMS = 8;
constexpr int RG_TILE = RG_THREADS * RG_ITEMS;

// compact summary for the cross-epoch conflict test: per category the owner of
// its earliest item (or none) and whether a second owner exists
struct Adj {
    uint32_t own[3];
    uint32_t multi;   // bit c: category c has two or more owners
};

__device__ __forceinline__ Adj adj_of(const Top2 &s) {
    Adj a;
    a.multi = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        a.own[c] = s.a[c] == EMPTY ? 0xFFFFFFFFu : (uint32_t)s.a[c];
        if (s.b[c] != EMPTY) a.multi |= 1u << c;
    }
    return a;
}

__device__ __forceinline__ bool adj_conflict(const Adj &P, const Adj &Q) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        if (P.own[i] == 0xFFFFFFFFu) continue;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (Q.own[j] == 0xFFFFFFFFu) continue;
            if ((i == 0 && j == 0) || (i == 2 && j == 2)) continue;   // read/read, atomic/atomic
            if (((P.multi >> i) & 1u) || ((Q.multi >> j) & 1u) || P.own[i] != Q.own[j]) return true;
        }
    }
    return false;
}

// Warp-aware traces (Theorem 1 with its warp conditions): a pair of one warp conflicts only when both
// are plain writes of the same statement or either came after divergence. The top-2 summary does not
// carry warps and statements, so these groups are searched pair by pair, as the definition reads.
__device__ __forceinline__ bool wa_conflict(uint32_t ap, uint32_t gp, uint32_t sp, uint32_t aq, uint32_t gq,
                                            uint32_t sq, uint32_t bt) {
    if (gp == gq) return false;
    const bool mp = ap != ACT_R, mq = aq != ACT_R;
    if (!mp && !mq) return false;
    if (ap == ACT_A && aq == ACT_A) return false;
    if (gp / bt == gq / bt && ((gp % bt) >> 5) == ((gq % bt) >> 5)) {
        const bool same_statement_writes = ap == ACT_W && aq == ACT_W && (sp & ~STMT_DIVERGED) == (sq & ~STMT_DIVERGED);
        if (!same_statement_writes && !(sp & STMT_DIVERGED) && !(sq & STMT_DIVERGED)) return false;
    }
    return true;
}

// one element of a warp-aware group: action, thread (block * bt + tid), statement word, visit order
struct WaItem {
    uint32_t act, gtid, stmt, vo;
};
__device__ __forceinline__ WaItem wa_item(const TraceDesc &d, uint64_t v) {
    const uint32_t idx = (uint32_t)v;   // the record index (warp-aware elements)
    return WaItem{payload_act(v), (uint32_t)(v >> 32) & 0x3FFFFFFFu, d.stmt[idx], d.events[idx].y};
}

// 64-bit minimum over the warp (all lanes take part)
__device__ __forceinline__ uint64_t warp_min64(uint64_t x) {
    const uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(x >> 32));
    const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(x >> 32) == hi ? (uint32_t)x : 0xFFFFFFFFu);
    return ((uint64_t)hi << 32) | lo;
}

// Races of group [gs, ge) of a warp-aware trace and the adjacency test against the group of the next epoch,
// if present. The stream does not hold a group's elements in schedule order (the record reads place their
// tiles in the order they finish), so every pair is examined and, per class, the lowest in schedule order
// kept: the pair whose later access comes first, then the earliest partner (schedule order: visit order,
// then record index). Called by one thread (lanes = 1) or by all lanes of a warp (lanes = 32), which share
// the work.
// Groups of up to WA_CACHE elements searched by one thread keep their items in registers: each item is
// gathered through its record index once, not once per pair (most groups hold 2-4 accesses). Item
// words: action << 30 | thread, statement word, visit order, record index.
constexpr uint32_t WA_CACHE = 3;

template <class K>
__device__ void wa_group(const K *__restrict__ keys, const uint64_t *__restrict__ vals, uint64_t gs, uint64_t ge,
                         uint64_t n, K kg, const TraceDesc &d, const Layout &L, const RaceStage &rs, Ctl *ctl,
                         uint32_t *nonred, uint32_t trace, uint32_t space, uint32_t block, uint32_t epoch,
                         uint32_t unit, int lane, int lanes) {
    uint64_t bq[2] = {EMPTY, EMPTY}, bp[2] = {EMPTY, EMPTY};   // (visit order << 32 | record index) of q and p
    // keep the pair (p, q) when it conflicts and is lower in its class than the one kept
    auto consider = [&](const WaItem &p, uint64_t kp, const WaItem &q, uint64_t kq) {
        if (kp >= kq || !wa_conflict(p.act, p.gtid, p.stmt, q.act, q.gtid, q.stmt, d.bt)) return;
        const int cls = (p.act != ACT_R && q.act != ACT_R) ? 0 : 1;
        if (kq < bq[cls] || (kq == bq[cls] && kp < bp[cls])) {
            bq[cls] = kq;
            bp[cls] = kp;
        }
    };
    const uint32_t g = (uint32_t)min(ge - gs, (uint64_t)WA_CACHE + 1u);
    const bool cached = lanes == 1 && g <= WA_CACHE;
    uint32_t c_ag[WA_CACHE] = {}, c_st[WA_CACHE] = {}, c_vo[WA_CACHE] = {}, c_ix[WA_CACHE] = {};
    auto c_item = [&](int i) { return WaItem{c_ag[i] >> 30, c_ag[i] & 0x3FFFFFFFu, c_st[i], c_vo[i]}; };
    auto c_key = [&](int i) { return ((uint64_t)c_vo[i] << 32) | c_ix[i]; };
    if (cached) {
#pragma unroll
        for (int i = 0; i < (int)WA_CACHE; i++) {
            c_ag[i] = c_st[i] = c_vo[i] = c_ix[i] = 0u;
            if ((uint32_t)i < g) {
                const uint64_t v = vals[gs + i];
                const WaItem it = wa_item(d, v);
                c_ag[i] = (it.act << 30) | it.gtid;
                c_st[i] = it.stmt;
                c_vo[i] = it.vo;
                c_ix[i] = (uint32_t)v;
            }
        }
#pragma unroll
        for (int a = 0; a < (int)WA_CACHE; a++)
#pragma unroll
            for (int b = 0; b < (int)WA_CACHE; b++)
                if ((uint32_t)a < g && (uint32_t)b < g) consider(c_item(b), c_key(b), c_item(a), c_key(a));
    } else {
        for (uint64_t qi = gs + lane; qi < ge; qi += lanes) {
            const WaItem q = wa_item(d, vals[qi]);
            const uint64_t kq = ((uint64_t)q.vo << 32) | (uint32_t)vals[qi];
            for (uint64_t pi = gs; pi < ge; pi++) {
                const WaItem p = wa_item(d, vals[pi]);
                consider(p, ((uint64_t)p.vo << 32) | (uint32_t)vals[pi], q, kq);
            }
        }
    }
#pragma unroll
    for (int cls = 0; cls < 2; cls++) {
        if (lanes > 1) {
            const uint64_t mq = warp_min64(bq[cls]);
            bp[cls] = warp_min64(bq[cls] == mq ? bp[cls] : EMPTY);
            bq[cls] = mq;
        }
        if (lane == 0 && bq[cls] != EMPTY) {
            const uint32_t ip = (uint32_t)bp[cls], iq = (uint32_t)bq[cls];
            const uint4 ep = d.events[ip], eq = d.events[iq];
            const uint32_t gp = ep.z * d.bt + (ep.w & 0xFFFFu), gq = eq.z * d.bt + (eq.w & 0xFFFFu);
            emit_race(rs, ctl, trace, race_key(L, trace, space, 0u, block, epoch, unit, (uint32_t)cls),
                      ((uint64_t)ep.y << 32) | gp, ((uint64_t)eq.y << 32) | gq);
        }
    }
    // barrier `epoch` is needed when a pair across this group and the next epoch's group conflicts
    if (ge < n && keys[ge] == kg + 1) {
        bool needed = false;
        for (uint64_t qi = ge; qi < n && keys[qi] == kg + 1 && !needed; qi++) {
            const WaItem q = wa_item(d, vals[qi]);
            if (cached) {
#pragma unroll
                for (int b = 0; b < (int)WA_CACHE; b++)
                    if ((uint32_t)b < g && !needed) {
                        const WaItem p = c_item(b);
                        needed = wa_conflict(p.act, p.gtid, p.stmt, q.act, q.gtid, q.stmt, d.bt);
                    }
            } else {
                for (uint64_t pi = gs + lane; pi < ge && !needed; pi += lanes) {
                    const WaItem p = wa_item(d, vals[pi]);
                    needed = wa_conflict(p.act, p.gtid, p.stmt, q.act, q.gtid, q.stmt, d.bt);
                }
            }
            if (lanes > 1) needed = __any_sync(0xFFFFFFFFu, needed);
        }
        if (needed && lane == 0) mark_needed_once(nonred, L, block, epoch);
    }
}

constexpr uint32_t RG_LONG = 32;                             // segments longer than this are reduced by a warp
constexpr uint32_t RG_MAX_LONG = RG_TILE / (RG_LONG + 1) + 1;  // long segments a tile can hold
constexpr uint32_t RG_HAS_HEAD = 1u, RG_PREV_HEAD = 2u;

// What a tile publishes for the tiles after it.
struct RgTile {
    Top2 last;        // its last piece: from its last head (or, without a head, its first element) to its end
    Top2 prev;        // the piece before its last head: from the head before that (RG_PREV_HEAD) or its start
    uint32_t head;    // element index of its last head (RG_HAS_HEAD)
    uint32_t flags;
};

template <class K, bool INTER>
constexpr size_t reduce_groups_smem() {
    return (size_t)RG_TILE * (8 + sizeof(K)) + (INTER ? 0 : (RG_TILE + 1) * sizeof(Adj)) + (RG_TILE + 2) * 2;
}

// The top-2 summary of the union of the lanes' summaries, in every lane. Per category the first item is
// the smallest first item; the second is the smallest item of another owner than the first's: a lane's
// first item when its owner differs, else the lane's second item (which has another owner than the lane's
// first, that is than the union's first).
template <class Own>
__device__ __forceinline__ void top2_warp_merge(Top2 &s, const Own &own) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const uint64_t a = warp_min64(s.a[c]);
        const uint64_t cand = (s.a[c] != EMPTY && own(s.a[c]) != own(a)) ? s.a[c] : s.b[c];
        s.b[c] = warp_min64(cand);
        s.a[c] = a;
    }
}

// the union of every thread's summary, in every thread (all threads of the CTA call it)
template <class Own>
__device__ __forceinline__ Top2 top2_cta_merge(Top2 s, const Own &own, Top2 *s_part) {
    top2_warp_merge(s, own);
    __syncthreads();   // s_part is free
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    Top2 r;
    if ((threadIdx.x & 31) < RG_THREADS / 32) r = s_part[threadIdx.x & 31];
    else r.clear();
    top2_warp_merge(r, own);
    return r;
}

__device__ __forceinline__ Top2 ldcg_top2(const Top2 *p) {
    const unsigned long long *q = reinterpret_cast<const unsigned long long *>(p);
    Top2 s;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        s.a[c] = __ldcg(q + c);
        s.b[c] = __ldcg(q + 3 + c);
    }
    return s;
}

// Wait until tile j of this launch has published. False when the wait gave up (ctl->timeout is then set,
// which stops every other waiter too).
__device__ __forceinline__ bool rg_wait(const uint32_t *ready, uint64_t j, uint32_t tag, Ctl *ctl, uint64_t wait_ns) {
    const volatile uint32_t *r = ready + j;
    if (*r != tag) {
        const uint64_t t0 = globaltimer_ns();
        for (uint32_t i = 1; *r != tag; i++) {
            if ((i & 63) == 0) {
                if (*(volatile unsigned int *)&ctl->timeout) return false;
                if (globaltimer_ns() - t0 > wait_ns) {
                    atomicExch(&ctl->timeout, 1u);
                    return false;
                }
            }
        }
    }
    __threadfence();
    return true;
}

// shared scratch of a look-back
struct RgLook {
    Top2 acc;
    uint32_t head, ok, found, first[RG_THREADS / 32];
    uint64_t htile;
};

// The summary of the group open at the end of tile j0, from its head to the end of j0: the last pieces that
// tiles j0, j0-1, ... published, down to the first of them that has a head. All threads of the CTA call it
// and receive the summary, the element index of the group's head and the tile holding it; false (in all
// threads) when a wait gave up.
template <class Own>
__device__ bool rg_lookback(uint64_t j0, const RgTile *pub, const uint32_t *ready, uint32_t tag, Ctl *ctl,
                            uint64_t wait_ns, const Own &own, Top2 *s_part, RgLook &lk, Top2 &S, uint32_t &head,
                            uint64_t &htile) {
    const int tid = threadIdx.x;
    if (tid == 0) {   // most groups began in the tile just before
        lk.ok = rg_wait(ready, j0, tag, ctl, wait_ns) ? 1u : 0u;
        lk.found = 0;
        if (lk.ok) {
            lk.acc = ldcg_top2(&pub[j0].last);
            if (__ldcg(&pub[j0].flags) & RG_HAS_HEAD) {
                lk.found = 1;
                lk.head = __ldcg(&pub[j0].head);
                lk.htile = j0;
            }
        }
    }
    __syncthreads();
    if (!lk.ok) return false;
    int64_t base = (int64_t)j0 - 1;
    while (!lk.found && base >= 0) {
        // tiles base, base - 1, ..., base - 255: one per thread
        const int64_t j = base - tid;
        bool ok = true, hh = false;
        if (j >= 0) {
            ok = rg_wait(ready, (uint64_t)j, tag, ctl, wait_ns);
            if (ok) hh = (__ldcg(&pub[j].flags) & RG_HAS_HEAD) != 0u;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hh);
        if ((tid & 31) == 0) lk.first[tid >> 5] = bal ? (uint32_t)(tid + __ffs(bal) - 1) : (uint32_t)RG_THREADS;
        if (__syncthreads_or(!ok)) return false;
        uint32_t first = RG_THREADS;   // the thread of the nearest tile with a head
#pragma unroll
        for (int w = 0; w < RG_THREADS / 32; w++) first = min(first, lk.first[w]);
        Top2 part;
        part.clear();
        if (j >= 0 && (uint32_t)tid <= first) part = ldcg_top2(&pub[j].last);
        part = top2_cta_merge(part, own, s_part);
        if (tid == 0) {
            top2_merge(lk.acc, part, own);
            if (first < (uint32_t)RG_THREADS) {
                lk.found = 1;
                lk.htile = (uint64_t)(base - first);
                lk.head = __ldcg(&pub[lk.htile].head);
            }
        }
        __syncthreads();
        base -= RG_THREADS;
    }
    S = lk.acc;
    head = lk.head;
    htile = lk.htile;
    __syncthreads();   // lk is free again
    return true;
}

// the group before one of key kq (ended right before its head) is the same unit's previous epoch: its
// key is kq - 1, or (the paper's visit-order counters) any key of the same block and unit
template <class K>
__device__ __forceinline__ bool rg_adjacent(K kp, K kq, const Layout &L, const TraceDesc *td, const uint32_t *tob,
                                            uint32_t bu) {
    if (kq == kp + 1) return true;
    const uint32_t be = L.be;
    if (((uint64_t)kq >> be) != ((uint64_t)kp >> be)) return false;
    return (td[tob[(uint64_t)kp >> (bu + be)]].flags & TF_PAPER_ORDER) != 0;
}

template <class K, bool INTER>
__global__ void __launch_bounds__(RG_THREADS)
k_reduce_groups(const K *__restrict__ keys, const uint64_t *__restrict__ vals, const uint32_t *n_ptr, uint64_t n_max,
                Layout L, const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, uint32_t space,
                uint32_t bu, Ctl *ctl, uint32_t *nonred, RaceStage rs, RgTile *pub, uint32_t *ready, uint32_t tag,
                uint32_t *tile_ctr, uint64_t wait_ns) {
    extern __shared__ __align__(16) uint8_t rg_smem[];
    uint64_t *sval = reinterpret_cast<uint64_t *>(rg_smem);
    K *skey = reinterpret_cast<K *>(rg_smem + RG_TILE * 8);
    Adj *sadj = reinterpret_cast<Adj *>(rg_smem + RG_TILE * (8 + sizeof(K)));
    uint16_t *shead = reinterpret_cast<uint16_t *>(rg_smem + RG_TILE * (8 + sizeof(K)) +
                                                   (INTER ? 0 : (RG_TILE + 1) * sizeof(Adj)));
    __shared__ uint32_t wsum[RG_THREADS / 32];
    __shared__ Top2 s_part[RG_THREADS / 32];
    __shared__ Top2 s_first, s_last, s_prev;   // segment 0, the last segment, the segment before it
    __shared__ RgLook s_look;
    __shared__ uint16_t s_long[RG_MAX_LONG];
    __shared__ uint32_t s_G, s_nlong, s_ends, s_stop;
    __shared__ uint64_t s_tile;
    // (block << 12 | barrier) + 1 of the needed-barrier marks this CTA has sent: a tile's groups are of one
    // or two blocks, so most marks repeat one this CTA sent already and skip even the read of the word
    __shared__ uint32_t s_mk[256];
    for (int i = threadIdx.x; i < 256; i += RG_THREADS) s_mk[i] = 0;
    auto mark = [&](uint32_t block, uint32_t k) {
        if (block < (1u << 20) && k < 4096u) {
            const uint32_t key = ((block << 12) | k) + 1u, h = (key * 0x9E3779B1u) >> 24;
            if (*(volatile uint32_t *)&s_mk[h] == key) return;
            s_mk[h] = key;
        }
        mark_needed_once(nonred, L, block, k);
    };
    const uint64_t n = min((uint64_t)*n_ptr, n_max);
    const uint64_t ntiles = (n + RG_TILE - 1) / RG_TILE;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t be = L.be;
    const uint64_t umask = (bu >= 64) ? ~0ull : ((1ull << bu) - 1);
    const OwnThread own_t;
    auto own_of = [&](K kg) -> OwnBlock {   // inter-block owners: the blocks of the key's trace
        const uint32_t trace = (uint32_t)((uint64_t)kg >> (L.bug + L.bxr));
        return OwnBlock{td[trace].bt, td[trace].nb <= (1u << 20)};
    };
    // races of a finished group (and, intra streams, its adjacency summary), by one thread (lanes = 1) or
    // by all lanes of a warp holding the same summary (lanes = 32)
    auto finish = [&](K kg, uint64_t gs, uint64_t ge, const Top2 &S, Adj *adj_out, int ln, int lanes) {
        if (INTER) {
            if (ln != 0) return;
            const uint32_t trace = (uint32_t)((uint64_t)kg >> (L.bug + L.bxr));
            const OwnBlock own_b = own_of(kg);
            const uint32_t unit = (uint32_t)((uint64_t)kg & umask);
            // the visit order of a paper-counter trace's group (0 for other traces)
            const uint32_t vord = (uint32_t)(((uint64_t)kg >> L.bug) & ((1ull << L.bxr) - 1));
#pragma unroll
            for (int cls = 0; cls < 2; cls++) {
                uint64_t p, q;
                if (!lowest_pair(S, cls, own_b, p, q)) continue;
                // owner codes back to block * block_threads + tid
                p = (p & ~0xFFFFFFFFull) | own_b.gtid((uint32_t)p);
                q = (q & ~0xFFFFFFFFull) | own_b.gtid((uint32_t)q);
                emit_race(rs, ctl, trace, race_key(L, trace, 1u, 1u, 0u, vord, unit, cls), p, q);
            }
        } else {
            const uint32_t trace = tob[(uint64_t)kg >> (bu + be)];
            const uint64_t sk = (uint64_t)kg >> be;
            const uint32_t block = (uint32_t)(sk >> bu), unit = (uint32_t)(sk & umask);
            const uint32_t epoch = (uint32_t)((uint64_t)kg & ((1ull << be) - 1));
            const TraceDesc &d = td[trace];
            if (d.flags & TF_WARP_AWARE) {
                // pair by pair, with the adjacency test against the next epoch's group
                wa_group(keys, vals, gs, ge, n, kg, d, L, rs, ctl, nonred, trace, space, block, epoch, unit, ln, lanes);
                if (ln == 0) {
                    Top2 none;
                    none.clear();
                    *adj_out = adj_of(none);
                }
            } else if (ln == 0) {
                emit_group(L, rs, ctl, S, own_t, trace, space, 0u, block, epoch, unit);
                *adj_out = adj_of(S);
            }
        }
    };
    auto warp_aware = [&](K kg) -> bool {
        return !INTER && (td[tob[(uint64_t)kg >> (bu + be)]].flags & TF_WARP_AWARE) != 0;
    };
    for (;;) {
        if (tid == 0) {
            s_tile = atomicAdd(tile_ctr, 1u);
            s_stop = must_stop(ctl) ? 1u : 0u;
            s_nlong = 0;
        }
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles || s_stop) break;
        const uint64_t t0 = tile * RG_TILE;
        const uint32_t m = (uint32_t)min((uint64_t)RG_TILE, n - t0);
        for (uint32_t i = tid; i < m; i += RG_THREADS) {
            skey[i] = keys[t0 + i];
            sval[i] = vals[t0 + i];
        }
        __syncthreads();
        // heads among the elements [tid*8, tid*8+8)
        uint32_t hm = 0;
        const K kprev0 = (t0 > 0) ? keys[t0 - 1] : K(0);
#pragma unroll
        for (int j = 0; j < RG_ITEMS; j++) {
            const uint32_t i = tid * RG_ITEMS + j;
            if (i < m) {
                const bool h = (t0 + i == 0) || (i == 0 ? skey[0] != kprev0 : skey[i] != skey[i - 1]);
                hm |= (h ? 1u : 0u) << j;
            }
        }
        const uint32_t nh = __popc(hm);
        const uint32_t hbase = block_excl_scan_256(nh, wsum);
        {
            uint32_t o = hbase;
#pragma unroll
            for (int j = 0; j < RG_ITEMS; j++)
                if ((hm >> j) & 1u) shead[o++] = (uint16_t)(tid * RG_ITEMS + j);
        }
        if (tid == RG_THREADS - 1) s_G = hbase + nh;   // heads in this tile
        if (tid == 0) s_ends = (t0 + m >= n || keys[t0 + m] != skey[m - 1]) ? 1u : 0u;   // the last piece ends here
        __syncthreads();
        const uint32_t G = s_G;
        const bool ends = s_ends != 0u;
        const uint32_t fhead = G ? shead[0] : m;
        // Segments: 0 = [0, first head), s = 1..G = [head s-1, head s or the tile end). Segments 1..G-1 are
        // groups inside the tile; segment G is finished here when the tile ends it; segment 0 (when not empty)
        // ends a group that began before, finished after the look-back.
        auto segment_done = [&](uint32_t s, uint32_t a, uint32_t e, const Top2 &S, int ln, int lanes) {
            if (s == 0) {
                if (ln == 0) s_first = S;
                return;
            }
            if (ln == 0 && s == G) s_last = S;
            if (ln == 0 && s + 1 == G && G >= 2) s_prev = S;
            if (s < G || ends) finish(skey[a], t0 + a, t0 + e, S, INTER ? nullptr : &sadj[s], ln, lanes);
        };
        for (uint32_t s = tid; s <= G; s += RG_THREADS) {
            const uint32_t a = s == 0 ? 0u : shead[s - 1], e = s < G ? shead[s] : m;
            if (a == e) continue;   // segment 0 of a tile that starts with a head
            if (e - a > RG_LONG) {
                s_long[atomicAdd(&s_nlong, 1u)] = (uint16_t)s;
                continue;
            }
            Top2 S;
            S.clear();
            if (INTER) {
                const OwnBlock own_b = own_of(skey[a]);
                for (uint32_t j = a; j < e; j++) top2_add(S, payload_act(sval[j]), payload_item(sval[j]), own_b);
            } else {
                for (uint32_t j = a; j < e; j++) top2_add(S, payload_act(sval[j]), payload_item(sval[j]), own_t);
            }
            segment_done(s, a, e, S, 0, 1);
        }
        __syncthreads();
        // long segments: a warp each, lanes striding, then a warp-wide merge
        const uint32_t nlong = s_nlong;
        for (uint32_t q = warp; q < nlong; q += RG_THREADS / 32) {
            const uint32_t s = s_long[q];
            const uint32_t a = s == 0 ? 0u : shead[s - 1], e = s < G ? shead[s] : m;
            Top2 S;
            S.clear();
            if (INTER) {
                const OwnBlock own_b = own_of(skey[a]);
                for (uint32_t j = a + lane; j < e; j += 32) top2_add(S, payload_act(sval[j]), payload_item(sval[j]), own_b);
                top2_warp_merge(S, own_b);
            } else {
                for (uint32_t j = a + lane; j < e; j += 32) top2_add(S, payload_act(sval[j]), payload_item(sval[j]), own_t);
                top2_warp_merge(S, own_t);
            }
            segment_done(s, a, e, S, lane, 32);   // every lane holds the merged summary
        }
        __syncthreads();
        // publish for the tiles after this one
        if (tid == 0) {
            RgTile &P = pub[tile];
            Top2 prev;
            prev.clear();
            uint32_t flags = 0, head = 0;
            if (G) {
                flags |= RG_HAS_HEAD;
                head = (uint32_t)(t0 + shead[G - 1]);
                if (G >= 2) {
                    prev = s_prev;
                    flags |= RG_PREV_HEAD;
                } else if (fhead > 0) {
                    prev = s_first;
                }
            }
            P.last = G ? s_last : s_first;
            P.prev = prev;
            P.head = head;
            P.flags = flags;
            __threadfence();
            *(volatile uint32_t *)&ready[tile] = tag;
        }
        // the group that ends in segment 0 began in an earlier tile; intra streams also need the summary of
        // the group that ended right before this tile (the predecessor of segment 1)
        const bool fin0 = fhead > 0 && (G > 0 || ends);
        if (tile > 0 && (fin0 || (!INTER && fhead == 0 && G > 0))) {
            Top2 LB;
            uint32_t lb_head = 0;
            uint64_t lb_tile = 0;
            const K k0 = skey[0];
            bool ok;
            if (INTER) ok = rg_lookback(tile - 1, pub, ready, tag, ctl, wait_ns, own_of(k0), s_part, s_look, LB, lb_head, lb_tile);
            else ok = rg_lookback(tile - 1, pub, ready, tag, ctl, wait_ns, own_t, s_part, s_look, LB, lb_head, lb_tile);
            if (!ok) break;
            if (fin0) {
                if (warp == 0) {   // the first warp finishes it (a warp-aware group's pairs are shared out)
                    if (INTER) top2_merge(LB, s_first, own_of(k0));
                    else top2_merge(LB, s_first, own_t);
                    finish(k0, lb_head, t0 + fhead, LB, INTER ? nullptr : &sadj[0], lane, 32);
                }
                if (!INTER && lb_head > 0 && !warp_aware(k0)) {
                    // the group before it: the piece before the last head of the head's tile, and what
                    // came before that piece when it did not start at a head
                    Top2 P = ldcg_top2(&pub[lb_tile].prev);
                    const uint32_t pf = __ldcg(&pub[lb_tile].flags);
                    if (!(pf & RG_PREV_HEAD)) {
                        Top2 X;
                        uint32_t xh;
                        uint64_t xt;
                        if (!rg_lookback(lb_tile - 1, pub, ready, tag, ctl, wait_ns, own_t, s_part, s_look, X, xh, xt)) break;
                        top2_merge(P, X, own_t);
                    }
                    __syncthreads();   // sadj[0] is written
                    if (tid == 0) {
                        const K kp = keys[lb_head - 1];
                        if (rg_adjacent(kp, k0, L, td, tob, bu) && adj_conflict(adj_of(P), sadj[0]))
                            mark((uint32_t)(((uint64_t)kp >> be) >> bu), (uint32_t)((uint64_t)kp & ((1ull << be) - 1)));
                    }
                }
            } else if (!INTER && tid == 0) {
                if (warp_aware(kprev0)) {
                    Top2 none;
                    none.clear();
                    sadj[0] = adj_of(none);
                } else {
                    sadj[0] = adj_of(LB);
                }
            }
        }
        __syncthreads();
        // intra streams: each group finished inside the tile against the group before it
        if (!INTER && G > 0) {
            const uint32_t last_fin = ends ? G : G - 1;
            for (uint32_t s = 1 + tid; s <= last_fin; s += RG_THREADS) {
                const uint32_t a = shead[s - 1];
                if (t0 + a == 0) continue;   // the stream's first group
                const K kq = skey[a], kp = a > 0 ? skey[a - 1] : kprev0;
                if (rg_adjacent(kp, kq, L, td, tob, bu) && adj_conflict(sadj[s - 1], sadj[s]))
                    mark((uint32_t)(((uint64_t)kp >> be) >> bu), (uint32_t)((uint64_t)kp & ((1ull << be) - 1)));
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Outputs
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t race_trace(const Layout &L, uint64_t k) {
    const uint32_t s = 3 + L.bu + L.be + L.bb;
    return s >= 64 ? 0u : (uint32_t)(k >> s);
}

// Drop the hash path's races of blocks that fell back to the sort path (which
// emits them again), keep the rest in any order, and build the digit
// histograms of the kept keys for the canonical sort.
__global__ void __launch_bounds__(256)
k_race_filter(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ idx, uint64_t *okeys, uint64_t *oidx,
              Layout L, const uint32_t *__restrict__ binel, TState *ts, Ctl *ctl, uint32_t *hist) {
    __shared__ uint32_t sh[8 * RADIX];
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t s_base;
    const int tid = threadIdx.x;
    if (must_stop(ctl)) return;
    for (int i = tid; i < 8 * RADIX; i += 256) sh[i] = 0;
    __syncthreads();
    const uint64_t n = min((uint64_t)*(volatile unsigned int *)&ctl->n_races, L.race_cap);
    const uint64_t bmask = (1ull << L.bb) - 1;
    for (uint64_t base = (uint64_t)blockIdx.x * 256; base < n; base += (uint64_t)gridDim.x * 256) {
        const uint64_t i = base + tid;
        bool keep = false;
        uint64_t k = 0, ix = 0;
        if (i < n) {
            k = keys[i];
            ix = idx[i];
            keep = true;
            if (ix & RACE_FROM_HASH) {
                ix &= ~RACE_FROM_HASH;
                const uint32_t t = race_trace(L, k);
                const uint64_t blk = (k >> (1 + L.bu + L.be)) & bmask;
                if (t >= L.T || blk >= L.NB || binel[blk] != 0 || *(volatile unsigned int *)&ts[t].inel != 0) {
                    keep = false;
                    if (t < L.T) atomicSub(&ts[t].n_races, 1u);
                }
            }
            if (keep)
                for (uint32_t q = 0; q < L.np_r; q++) atomicAdd(&sh[q * RADIX + digit_of(k, q)], 1u);
        }
        const uint32_t pre = block_excl_scan_256(keep ? 1u : 0u, wsum);
        if (tid == 255) s_base = atomicAdd(&ctl->n_rf, pre + (keep ? 1u : 0u));
        __syncthreads();
        if (keep) {
            okeys[s_base + pre] = k;
            oidx[s_base + pre] = ix;
        }
        __syncthreads();
    }
    __syncthreads();
    for (int i = tid; i < (int)(L.np_r * RADIX); i += 256)
        if (sh[i]) atomicAdd(&hist[(L.p0_r + i / RADIX) * RADIX + (i % RADIX)], sh[i]);
}

// first position of each trace in the sorted race list
__global__ void k_race_starts(const uint64_t *__restrict__ keys, Layout L, Ctl *ctl, TState *ts) {
    if (must_stop(ctl)) return;
    const uint64_t n = min((uint64_t)ctl->n_rf, L.race_cap);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = race_trace(L, keys[i]);
        if (t < L.T && (i == 0 || race_trace(L, keys[i - 1]) != t)) ts[t].race_start = (uint32_t)i;
    }
}

__global__ void k_write_races(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ idx,
                              const uint4 *__restrict__ pay, Layout L, const TraceDesc *td, TState *ts, Ctl *ctl) {
    if (must_stop(ctl)) return;
    const uint64_t n = min((uint64_t)ctl->n_rf, L.race_cap);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const uint32_t t = race_trace(L, k);
        if (t >= L.T || trace_bad(ts[t])) continue;
        const TraceDesc &d = td[t];
        const uint64_t rank = i - ts[t].race_start;
        if (rank >= d.races_cap) continue;
        const uint64_t ix = idx[i];
        if (ix >= L.race_cap) continue;
        const uint4 p = pay[ix];
        const uint32_t cls = (uint32_t)(k & 1u);
        const uint32_t unit = (uint32_t)((k >> 1) & ((1ull << L.bu) - 1));
        uint32_t epoch = (uint32_t)((k >> (1 + L.bu)) & ((1ull << L.be) - 1));
        uint32_t block = (uint32_t)((k >> (1 + L.bu + L.be)) & ((1ull << L.bb) - 1)) - d.block_off;
        const uint32_t scope = (uint32_t)((k >> (1 + L.bu + L.be + L.bb)) & 1u);
        const uint32_t space = (uint32_t)((k >> (2 + L.bu + L.be + L.bb)) & 1u);
        if (scope) {   // inter-block: no block; the visit order of a paper-counter trace, else no epoch
            block = 0xFFFFFFFFu;
            if (!(d.flags & TF_PAPER_ORDER)) epoch = 0xFFFFFFFFu;
        }
        uint4 *o = reinterpret_cast<uint4 *>(d.races + 32 * rank);
        o[0] = make_uint4(space | (scope << 8) | (cls << 16), block, epoch, unit);
        o[1] = p;
    }
}

// per block: divergence flag and number of redundant barriers
__global__ void k_block_counts(const uint4 *stats, const uint32_t *nonred, Layout L, uint32_t *cnt_div,
                               uint32_t *cnt_red) {
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < L.NB; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 s = stats[b];
        cnt_div[b] = s.x != s.w ? 1u : 0u;
        uint32_t nr = 0;
        for (uint32_t wd = 0; wd < L.words; wd++) {
            const uint32_t lo = wd * 32;
            if (lo >= s.y) break;
            const uint32_t live = (s.y - lo >= 32) ? 0xFFFFFFFFu : ((1u << (s.y - lo)) - 1u);
            nr += __popc(~nonred[b * L.words + wd] & live);
        }
        cnt_red[b] = nr;
    }
}

// Single-CTA exclusive scan (1024 threads) of two count arrays of length m;
// oa[m], ob[m] receive the totals.
__global__ void __launch_bounds__(1024) k_scan2(const uint32_t *a, const uint32_t *b, uint64_t m, uint32_t *oa,
                                                uint32_t *ob, Ctl *ctl) {
    __shared__ uint32_t ws[2][32];
    __shared__ uint32_t carry[2];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) { carry[0] = 0; carry[1] = 0; }
    __syncthreads();
    for (uint64_t base = 0; base < m; base += 1024) {
        const uint64_t i = base + tid;
        uint32_t x = i < m ? a[i] : 0u, y = i < m ? b[i] : 0u;
        uint32_t sx = x, sy = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t tx = __shfl_up_sync(0xFFFFFFFFu, sx, o), ty = __shfl_up_sync(0xFFFFFFFFu, sy, o);
            if (lane >= o) { sx += tx; sy += ty; }
        }
        if (lane == 31) { ws[0][w] = sx; ws[1][w] = sy; }
        __syncthreads();
        if (w == 0) {
            uint32_t vx = ws[0][lane], vy = ws[1][lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t tx = __shfl_up_sync(0xFFFFFFFFu, vx, o), ty = __shfl_up_sync(0xFFFFFFFFu, vy, o);
                if (lane >= o) { vx += tx; vy += ty; }
            }
            ws[0][lane] = vx;
            ws[1][lane] = vy;
        }
        __syncthreads();
        const uint32_t px = (w ? ws[0][w - 1] : 0u) + sx - x + carry[0];
        const uint32_t py = (w ? ws[1][w - 1] : 0u) + sy - y + carry[1];
        if (i < m) { oa[i] = px; ob[i] = py; }
        __syncthreads();
        if (tid == 0) { carry[0] += ws[0][31]; carry[1] += ws[1][31]; }
        __syncthreads();
    }
    if (tid == 0) {
        oa[m] = carry[0];
        ob[m] = carry[1];
        ctl->n_div = carry[0];
        ctl->n_red = carry[1];
    }
}

__global__ void k_block_write(const uint4 *stats, const uint32_t *nonred, Layout L, const TraceDesc *td,
                              const uint32_t *tob, const TState *ts, const uint32_t *ofs_div, const uint32_t *ofs_red,
                              uint32_t want_div, uint32_t want_red) {
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < L.NB; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = tob[b];
        if (trace_bad(ts[t])) continue;
        const TraceDesc &d = td[t];
        const uint4 s = stats[b];
        const uint64_t lb = b - d.block_off;
        if (want_div && s.x != s.w) {
            const uint64_t r = ofs_div[b] - ofs_div[d.block_off];
            if (r < d.divs_cap) reinterpret_cast<uint4 *>(d.divs)[r] = make_uint4((uint32_t)lb, s.x, s.w, s.z);
        }
        if (!want_red) continue;
        uint64_t o = ofs_red[b] - ofs_red[d.block_off];
        for (uint32_t k = 0; k < s.y && o < d.reds_cap; k++)
            if (!((nonred[b * L.words + (k >> 5)] >> (k & 31)) & 1u))
                reinterpret_cast<uint2 *>(d.reds)[o++] = make_uint2((uint32_t)lb, k);
    }
}

// per trace: OR of the non-redundant bits and of "barrier exists" over its blocks
__global__ void k_grid_or(const uint4 *stats, const uint32_t *nonred, const uint32_t *tob, Layout L, uint32_t *gnr,
                          uint32_t *ghas) {
    const uint64_t tot = (uint64_t)L.NB * L.words;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = i / L.words;
        const uint32_t wd = (uint32_t)(i % L.words), lo = wd * 32, mx = stats[b].y;
        if (lo >= mx) continue;
        const uint32_t live = (mx - lo >= 32) ? 0xFFFFFFFFu : ((1u << (mx - lo)) - 1u);
        const uint64_t slot = (uint64_t)tob[b] * L.words + wd;
        const uint32_t nr = nonred[i] & live;
        if (nr) atomicOr(&gnr[slot], nr);
        atomicOr(&ghas[slot], live);
    }
}

// one CTA per trace: list every barrier k that exists in some block and is redundant in all
__global__ void __launch_bounds__(1024) k_grid_list(const uint32_t *gnr, const uint32_t *ghas, Layout L,
                                                    const TraceDesc *td, TState *ts) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    const uint32_t t = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    const uint32_t nk = L.words * 32;
    const uint32_t *nr = gnr + (uint64_t)t * L.words, *hs = ghas + (uint64_t)t * L.words;
    const uint64_t cap = td[t].grid_cap;
    for (uint32_t base = 0; base < nk; base += 1024) {
        const uint32_t k = base + tid;
        const bool red = k < nk && ((hs[k >> 5] >> (k & 31)) & 1u) && !((nr[k >> 5] >> (k & 31)) & 1u);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, red);
        if (lane == 0) ws[w] = __popc(bal);
        __syncthreads();
        uint32_t pre = carry;
        for (int i = 0; i < w; i++) pre += ws[i];
        pre += __popc(bal & lanemask_lt());
        if (red && pre < cap && !trace_bad(ts[t])) td[t].grid[pre] = k;
        __syncthreads();
        if (tid == 0) {
            uint32_t s = 0;
            for (int i = 0; i < 32; i++) s += ws[i];
            carry += s;
        }
        __syncthreads();
    }
    if (tid == 0) ts[t].n_grid = carry;
}

// final report per trace: status and true counts
struct ReportArgs {
    uint32_t want_races, want_div, want_red;
};

// A workspace below the worst case: some stream or the race staging received more elements than its
// capacity (the elements beyond it were dropped, so the results are incomplete).
__device__ __forceinline__ bool stream_overflow(const Ctl *ctl, const Layout &L) {
    const volatile Ctl *c = ctl;
    return c->n_s > L.cap_s || c->n_g > L.cap_s || c->n_xf > L.cap_x1 || c->n_x > L.x_cap || c->n_races > L.race_cap;
}

__global__ void k_report(const TraceDesc *td, const TState *ts, const uint32_t *ofs_div, const uint32_t *ofs_red,
                         Layout L, Ctl *ctl, ReportArgs a) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < L.T; t += gridDim.x * blockDim.x) {
        const TraceDesc &d = td[t];
        const volatile TState *v = &ts[t];
        int32_t status = 0;
        uint32_t kind = 0;
        uint64_t bad = 0, nr = 0, nd = 0, nred = 0, ng = 0;
        if (v->bad_cnt) {
            status = 2; kind = 1; bad = ~v->bad_cnt;
        } else if (v->bad_rec) {
            status = 2; kind = 0; bad = ~v->bad_rec;
        } else {
            if (a.want_races) nr = v->n_races;
            if (a.want_div) nd = ofs_div[d.block_off + d.nb] - ofs_div[d.block_off];
            if (a.want_red) { nred = ofs_red[d.block_off + d.nb] - ofs_red[d.block_off]; ng = v->n_grid; }
            if (*(volatile unsigned int *)&ctl->timeout) status = 5;
            else if (L.compact && stream_overflow(ctl, L)) status = 3;
            else if (nr > d.races_cap || nd > d.divs_cap || nred > d.reds_cap || ng > d.grid_cap) status = 4;
        }
        uint8_t *report = d.report;
        reinterpret_cast<int32_t *>(report)[0] = status;
        reinterpret_cast<uint32_t *>(report)[1] = kind;
        uint64_t *r64 = reinterpret_cast<uint64_t *>(report);
        r64[1] = bad;
        r64[2] = nr;
        r64[3] = nd;
        r64[4] = nred;
        r64[5] = ng;
    }
}

}  // namespace simk
