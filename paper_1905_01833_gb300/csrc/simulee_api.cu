// simulee_api.cu - host side of the check: argument checks, workspace layout,
// kernel orchestration and the C ABI declared in include/simulee.h.
//
// Pipeline of one check (all on the caller's stream, no host synchronisation):
//   1. zero the control block, histograms, bitmaps and look-back status words
//   2. k_block_stats      barrier counts: per-block min/max, count validation
//   3. (unsorted traces)   radix sort of (visit order, index) -> schedule ranks
//   4. k_ingest           validate records; route to streams S, G, X; digit histograms
//   5. k_onesweep x P     LSD radix sort of S (block,unit,epoch), G (block,unit,epoch), X (unit)
//   6. k_reduce_intra     S and G: per-group top-2 summaries, races, epoch adjacency
//      k_reduce_inter     X: per-unit top-2 summaries over blocks, inter-block races
//   7. race sort          radix sort of race records by canonical key, then copy out
//   8. block outputs      divergence and redundant-barrier lists by prefix sums
//   9. k_report           status and counts
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/simulee.h"
#include "check_kernels.cuh"
#include "hash_path.cuh"
#include "fitness.cuh"
#include "models.cuh"
#include "paper_order.cuh"
#include "sort.cuh"

using namespace simk;

struct simulee_ctx {
    int device;
    int sms;
    simulee_options opt;
    bool attrs_set;
    uint32_t last_launches;
    cudaEvent_t stage_ev[2 * SIMULEE_STAGES];
    bool stage_on;
    std::vector<const void *> attr_fns;   // kernels whose shared-memory attribute is set
    // replay of repeated identical calls: the arguments of the last call launched directly (seen_key),
    // and the launch sequence of a call seen twice in a row captured as a CUDA graph (graph_key)
    std::vector<uint8_t> seen_key, graph_key;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint32_t graph_launches = 0;
    uint32_t last_replayed = 0;   // the last check call was one graph launch
    ~simulee_ctx() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

namespace {

uint32_t bits_for(uint64_t count) {   // bits to hold values 0 .. count-1
    uint32_t b = 0;
    while (b < 64 && (1ull << b) < count) b++;
    return b;
}
uint32_t passes_for(uint32_t bits) { return (bits + RADIX_BITS - 1) / RADIX_BITS; }
size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Want {
    bool races, div, red;
};

constexpr uint32_t kMaxTraces = 1u << 20;

simulee_status check_trace_args(const simulee_trace *t) {
    if (!t) return SIMULEE_EINVAL;
    if (t->n_events > 0 && !t->events) return SIMULEE_EINVAL;
    if (!t->barrier_counts) return SIMULEE_EINVAL;
    if (t->n_events >= (1ull << 31)) return SIMULEE_EINVAL;
    if (t->n_blocks == 0 || t->block_threads == 0 || t->block_threads > 1024) return SIMULEE_EINVAL;
    if ((uint64_t)t->n_blocks * t->block_threads > (1ull << 30)) return SIMULEE_EINVAL;
    if (t->max_barriers > 4095) return SIMULEE_EINVAL;
    if (t->flags & ~(SIMULEE_FLAG_UNSORTED | SIMULEE_FLAG_WARP_AWARE | SIMULEE_FLAG_PAPER_ORDER)) return SIMULEE_EINVAL;
    if ((t->flags & SIMULEE_FLAG_WARP_AWARE) && (t->flags & SIMULEE_FLAG_PAPER_ORDER)) return SIMULEE_EINVAL;
    if (t->flags & SIMULEE_FLAG_WARP_AWARE) {
        if (t->flags & SIMULEE_FLAG_UNSORTED) return SIMULEE_EINVAL;
        if (t->n_events > 0 && (!t->stmt || ((uintptr_t)t->stmt & 3u) != 0)) return SIMULEE_EINVAL;
    }
    if (((uintptr_t)t->events & 15u) != 0 || ((uintptr_t)t->barrier_counts & 3u) != 0) return SIMULEE_EINVAL;
    return SIMULEE_OK;
}

// digits per tile in the look-back status array: the widest of the call's passes
uint32_t status_digits(const Layout &L) { return std::max<uint32_t>(RADIX, 1u << L.radix_bits); }

// How make_layout sizes the record streams and the race staging.
//   FULL:    for the worst case (every record on the sort path, every group racing): never overflows.
//   COMPACT: the query of a compact workspace: streams hold the records of traces that take the sort
//            path from the start plus a slack of max(n / 16, 65536) elements (all of n at most).
//   FIT:     the layout of a call: FULL when the caller's workspace holds it, else the largest slack
//            that fits the caller's workspace; a count beyond a capacity reports SIMULEE_ENOMEM.
enum class Sizing { FULL, COMPACT, FIT };

// Batch-wide bit layouts, pass counts and workspace offsets (a single trace is a batch of one).
// sort_all: every trace takes the sort path (the options force it). avail: the caller's workspace
// bytes (Sizing::FIT).
simulee_status make_layout(const simulee_trace *tr, uint32_t T, int sms, const simulee_options &opt, Layout &L,
                           Sizing sizing = Sizing::FULL, bool sort_all = false, size_t avail = 0) {
    memset(&L, 0, sizeof L);
    if (T == 0 || T > kMaxTraces) return SIMULEE_EINVAL;
    uint64_t n = 0, nb = 0, tiles = 0;
    uint32_t maxb = 0, su = 0, gu = 0, uns = 0, maxnb = 0, paper = 0;
    for (uint32_t i = 0; i < T; i++) {
        const simulee_trace &t = tr[i];
        if (t.n_blocks == 0 || t.block_threads == 0 || t.block_threads > 1024 || t.max_barriers > 4095 ||
            t.n_events >= (1ull << 31) || (uint64_t)t.n_blocks * t.block_threads > (1ull << 30))
            return SIMULEE_EINVAL;
        n += t.n_events;
        nb += t.n_blocks;
        tiles += (t.n_events + IN_TILE - 1) / IN_TILE;
        maxb = std::max(maxb, t.max_barriers);
        maxnb = std::max(maxnb, t.n_blocks);
        su = std::max(su, t.shared_units);
        gu = std::max(gu, t.global_units);
        uns |= t.flags & SIMULEE_FLAG_UNSORTED;
        paper |= (t.flags & SIMULEE_FLAG_PAPER_ORDER) ? 1u : 0u;
    }
    if (n >= (1ull << 31) || nb >= (1ull << 31)) return SIMULEE_EINVAL;
    L.n = n;
    L.T = T;
    L.NB = (uint32_t)nb;
    L.ntiles_in = tiles;
    L.maxb = maxb;
    L.any_unsorted = uns;
    L.bb = bits_for(L.NB);
    L.bus = bits_for(su);
    L.bug = bits_for(gu);
    L.be = bits_for((uint64_t)maxb + 1);
    L.bu = std::max(L.bus, L.bug);
    L.btr = bits_for(T);
    L.bits_s = L.bb + L.bus + L.be;
    L.bits_g = L.bb + L.bug + L.be;
    // inter-block keys: trace | visit order (paper counters only) | unit
    L.any_paper = paper;
    L.bxr = paper ? L.be : 0;
    L.bits_x = L.btr + L.bxr + L.bug;
    L.bits_r = 3 + L.bb + L.be + L.bu + L.btr;
    L.bits_q = 32 + L.btr;
    if (L.bits_s > 64 || L.bits_g > 64 || L.bits_x > 64 || L.bits_r > 64 || L.bits_q > 64) return SIMULEE_EINVAL;
    L.wide_s = L.bits_s > 32;
    L.wide_g = L.bits_g > 32;
    L.wide_x = L.bits_x > 32;
    L.wide_q = L.bits_q > 32;
    L.np_s = passes_for(L.bits_s);
    L.np_g = passes_for(L.bits_g);
    L.np_x = passes_for(L.bits_x);
    L.np_r = passes_for(L.bits_r);
    L.np_q = uns ? passes_for(L.bits_q) : 0;
    L.p0_s = 0;
    L.p0_g = L.p0_s + L.np_s;
    L.p0_x = L.p0_g + L.np_g;
    L.p0_r = L.p0_x + L.np_x;
    L.p0_q = L.p0_r + L.np_r;
    if (L.p0_q + L.np_q > MAX_PASSES || L.np_s + L.np_g + L.np_x > IN_MAXP) return SIMULEE_EINVAL;
    L.words = std::max<uint32_t>(1, (maxb + 31) / 32);
    const uint64_t n1 = std::max<uint64_t>(L.n, 1);
    L.sort_items = opt.sort_items ? opt.sort_items : 16u;
    L.radix_bits = opt.radix_bits ? opt.radix_bits : (uint32_t)RADIX_BITS;
    L.hb_cap_eighths = opt.hash_cap_eighths ? opt.hash_cap_eighths : 7u;
    L.hb_pool_div = opt.hash_pool_div ? opt.hash_pool_div : 3u;

    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
    // zeroed by every call: control block, per-trace state, bitmaps
    L.off_ctl = take(sizeof(Ctl));
    L.off_ts = take((size_t)T * sizeof(TState));
    L.off_nonred = take((size_t)L.NB * L.words * 4);
    L.off_gridnr = take((size_t)T * L.words * 4);
    L.off_gridhas = take((size_t)T * L.words * 4);
    L.off_hist = take((size_t)MAX_PASSES * RADIX * 4);
    L.off_binel = take((size_t)L.NB * 4);
    L.swords = maxb / 32 + 1;
    L.off_spill = take((size_t)L.NB * L.swords * 4);
    L.off_tflag = take((size_t)std::max<uint64_t>(L.ntiles_in, 1) * 4);
    L.off_bbins = take((size_t)2 * HB_LGROUPS * HB_BINS * 4);
    // histograms of passes over digits of another width than 8 bits: one region per stream (S, G, X,
    // races, schedule ranks)
    const size_t w_region = (size_t)5 * W_SLOT_PASSES * W_RADIX_MAX * 4;
    if (L.radix_bits != (uint32_t)RADIX_BITS) L.off_hw = take(w_region);
    L.zero_end = o;
    if (L.radix_bits != (uint32_t)RADIX_BITS) L.off_dw = take(w_region);
    L.off_bstart = take((size_t)L.NB * 4);
    L.off_blist = take((size_t)L.NB * 4);
    L.off_bgroup = take((size_t)L.NB);
    L.off_fbt = take((size_t)std::max<uint64_t>(L.ntiles_in, 1) * 4);
    // block signatures of global units: indexed directly (each trace's units after the previous
    // traces' ones) when all traces' global units together fit 2^28 slots, else by a hash of
    // (trace, unit) into a power-of-two table about the size of the batch (a collision only keeps
    // records that a direct table would have dropped)
    if (gu > 0) {
        uint64_t sum_gu = 0;
        for (uint32_t i = 0; i < T; i++) sum_gu += tr[i].global_units;
        if (sum_gu <= (1ull << 28)) {
            L.sig_direct = 1;
            L.sig_slots = sum_gu;
        } else {
            uint64_t m = 1u << 16;
            while (m < L.n && m < (1ull << 28)) m <<= 1;
            L.sig_slots = m;
        }
        L.sig_or = maxnb <= (1u << 15) ? 1u : 0u;
        L.off_sig = take(L.sig_slots * 4);
    }
    L.off_td = take((size_t)T * sizeof(TraceDesc));
    L.off_tob = take((size_t)L.NB * 4);
    L.off_stats = take((size_t)L.NB * 16);
    L.off_cnt_div = take((size_t)L.NB * 4);
    L.off_cnt_red = take((size_t)L.NB * 4);
    L.off_ofs_div = take((size_t)(L.NB + 1) * 4);
    L.off_ofs_red = take((size_t)(L.NB + 1) * 4);
    L.off_dbase = take((size_t)MAX_PASSES * RADIX * 4);
    if (uns) {
        L.off_rank = take(n1 * 4);
        L.off_p2v = take(n1 * 4);
    }
    const size_t ks = L.wide_s ? 8 : 4, kg = L.wide_g ? 8 : 4, kx = L.wide_x ? 8 : 4;
    // inter-block stream: every global record, plus the unused tails of the chunks of slots
    // the hash path's warps reserve (one partial chunk per warp that reserved any)
    // (32 warps per SM in either CTA shape, at most one SM's worth per block)
    // (two launches at most, one per CTA shape)
    const uint64_t hash_warps = (uint64_t)std::max(1, std::min<int>(sms, (int)std::max<uint32_t>(L.NB, 1))) * 32 * 2;
    L.x_cap = n1 + std::min<uint64_t>(hash_warps, n1) * HB_XCH;
    // The rest scales with three capacities (elements): cs for each intra-block stream S and G, cx for
    // the inter-block elements kept by the filter, cr for the race staging. The first inter-block
    // buffer always holds x_cap slots (the record read writes every global record there).
    const size_t fixed = o;
    auto lay = [&](uint64_t cs, uint64_t cx, uint64_t cr, Layout &M) -> size_t {
        size_t p = fixed;
        auto tk = [&](size_t bytes) { size_t r = p; p = align_up(p + bytes); return r; };
        M.cap_s = cs;
        M.cap_x1 = cx;
        M.race_cap = cr;
        const uint64_t sort_max = std::max<uint64_t>(std::max<uint64_t>(cs, cx), std::max<uint64_t>(cr, uns ? n1 : 0));
        const uint64_t tile = (uint64_t)OS_THREADS * M.sort_items;
        M.status_tiles = (sort_max + tile - 1) / tile;
        M.off_status = tk((size_t)M.status_tiles * status_digits(M) * 8);
        M.rg_tiles = (std::max<uint64_t>(cs, cx) + RG_TILE - 1) / RG_TILE + 1;
        M.off_rgpub = tk((size_t)M.rg_tiles * sizeof(RgTile));
        M.off_rgready = tk((size_t)M.rg_tiles * 4);
        for (int i = 0; i < 2; i++) {
            M.off_sk[i] = tk(cs * ks);
            M.off_sv[i] = tk(cs * 8);
            M.off_gk[i] = tk(cs * kg);
            M.off_gv[i] = tk(cs * 8);
            M.off_xk[i] = tk((i == 0 ? M.x_cap : cx) * kx);
            M.off_xv[i] = tk((i == 0 ? M.x_cap : cx) * 8);
            M.off_rk[i] = tk(cr * 8);
            M.off_rv[i] = tk(cr * 8);
        }
        M.off_rp = tk(cr * 16);
        return p;
    };
    // full capacities: every record in S or G, every global record kept, two races per record
    const uint64_t full_r = 2 * L.n + 2;
    // records of traces that take the sort path from the start: the streams hold all of them
    uint64_t n_sort = 0;
    for (uint32_t i = 0; i < T; i++)
        if (sort_all || (tr[i].flags & (SIMULEE_FLAG_UNSORTED | SIMULEE_FLAG_WARP_AWARE | SIMULEE_FLAG_PAPER_ORDER)))
            n_sort += tr[i].n_events;
    // the unsorted traces' schedule-rank sort runs in the race buffers over all records
    auto caps = [&](uint64_t slack, uint64_t &cs, uint64_t &cx, uint64_t &cr) {
        cs = std::min<uint64_t>(n1, n_sort + slack);
        cx = std::min<uint64_t>(L.x_cap, n_sort + slack);
        cr = std::min<uint64_t>(full_r, std::max<uint64_t>(2 * n_sort + slack + 2, uns ? n1 : 0));
    };
    Layout F = L;
    const size_t full_total = lay(n1, L.x_cap, full_r, F);
    uint64_t slack = n1;
    if (sizing == Sizing::COMPACT) {
        slack = std::min<uint64_t>(n1, std::max<uint64_t>(n1 / 16, 65536));
    } else if (sizing == Sizing::FIT && avail < full_total) {
        uint64_t cs, cx, cr;
        caps(0, cs, cx, cr);
        Layout M = L;
        if (lay(cs, cx, cr, M) > avail) return SIMULEE_ENOMEM;
        uint64_t lo = 0, hi = n1;   // the largest slack whose layout fits `avail`
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo + 1) / 2;
            caps(mid, cs, cx, cr);
            if (lay(cs, cx, cr, M) <= avail) lo = mid;
            else hi = mid - 1;
        }
        slack = lo;
    }
    if (slack >= n1) {
        L = F;
        L.total = full_total;
        L.compact = 0;
    } else {
        uint64_t cs, cx, cr;
        caps(slack, cs, cx, cr);
        L.total = lay(cs, cx, cr, L);
        L.compact = (cs < n1 || cx < L.x_cap || cr < full_r) ? 1u : 0u;
    }
    return SIMULEE_OK;
}

template <class K>
void set_sort_attr() {
    cudaFuncSetAttribute(k_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem<K>());
}

template <class KX, class SH>
void set_hash_attr() {
    cudaFuncSetAttribute(k_hash_blocks<KX, SH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)hash_blocks_smem<SH>());
    cudaFuncSetAttribute(k_hash_blocks<KX, SH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)hash_blocks_smem<SH>());
}

template <class K, bool INTER>
void set_reduce_attr() {
    cudaFuncSetAttribute(k_reduce_groups<K, INTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)reduce_groups_smem<K, INTER>());
}

// one-time opt-in to large dynamic shared memory, per kernel instantiation and context
template <class F>
bool attr_done(simulee_ctx *ctx, F *fn) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    for (const void *p : ctx->attr_fns)
        if (p == (const void *)fn) return true;
    ctx->attr_fns.push_back((const void *)fn);
    return false;
}

struct Run {
    simulee_ctx *ctx;
    cudaStream_t st;
    Layout L;
    uint8_t *ws;
    Ctl *ctl;
    uint64_t wait_ns;
    uint32_t withhold;   // applied to the first sort pass launched
    bool first_pass_done = false;
    uint32_t launches = 0;

    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }

    void mark(int stage, int end) const {
        if (ctx->stage_on) cudaEventRecord(ctx->stage_ev[2 * stage + end], st);
    }

    int sort_grid(uint64_t n_max, uint32_t bits) const {
        const uint64_t tile = (uint64_t)OS_THREADS * L.sort_items;
        const uint64_t tiles = (n_max + tile - 1) / tile;
        // the 11-bit passes hold one CTA per SM (their per-digit shared arrays)
        const uint64_t per_sm = bits > 8 ? 1u : (ctx->opt.sort_ctas_per_sm ? ctx->opt.sort_ctas_per_sm : 3u);
        return (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)ctx->sms * per_sm));
    }

    uint32_t wpass = 0;   // passes issued over digits of another width (their tile counters and tags)

    template <class K, int ITEMS, int BITS>
    void pass(int grid, const K *kin, const uint64_t *vin, K *kout, uint64_t *vout, const uint32_t *n_ptr,
              uint64_t n_max, uint32_t shift, const uint32_t *dbase, uint32_t tag, uint32_t *ctr, uint32_t tile_cap) {
        const uint32_t wh = first_pass_done ? 0u : withhold;
        first_pass_done = true;
        if (!attr_done(ctx, k_onesweep<K, ITEMS, BITS>))
            cudaFuncSetAttribute(k_onesweep<K, ITEMS, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem<K, ITEMS, BITS>());
        k_onesweep<K, ITEMS, BITS><<<grid, OS_THREADS, onesweep_smem<K, ITEMS, BITS>(), st>>>(
            kin, vin, kout, vout, n_ptr, n_max, shift, dbase, at<unsigned long long>(L.off_status), tag, ctr, ctl,
            wait_ns, wh, tile_cap);
        launches++;
    }

    // the passes of one sort over BITS-bit digits with tiles of 256 x ITEMS; 8-bit digits take their
    // histograms from the record reads (passes p0.. of the call), other widths count them first
    template <class K, int ITEMS, int BITS>
    int sort_w(size_t koff[2], size_t voff[2], const uint32_t *n_ptr, uint64_t n_max, uint32_t key_bits, uint32_t p0,
               int start, uint32_t tile_cap, uint32_t slot) {
        const uint32_t np = (key_bits + BITS - 1) / BITS;
        if (np == 0) return start;
        const int grid = sort_grid(n_max, BITS);
        const uint32_t *dbase;
        constexpr uint32_t R = 1u << BITS;
        if (BITS == RADIX_BITS) {
            dbase = at<uint32_t>(L.off_dbase) + (size_t)p0 * RADIX;
        } else {
            uint32_t *hw = at<uint32_t>(L.off_hw) + (size_t)slot * W_SLOT_PASSES * W_RADIX_MAX;
            uint32_t *dw = at<uint32_t>(L.off_dw) + (size_t)slot * W_SLOT_PASSES * W_RADIX_MAX;
            k_hist_keys<K, BITS><<<grid_for(n_max, (uint64_t)OS_THREADS * 16, 4), 256, np * R * 4, st>>>(
                at<K>(koff[start]), n_ptr, n_max, np, hw, ctl);
            k_digit_bases_w<BITS><<<np, OS_THREADS, 0, st>>>(hw, dw);
            launches += 2;
            dbase = dw;
        }
        for (uint32_t p = 0; p < np; p++) {
            const int src = (start + (int)p) & 1, dst = src ^ 1;
            uint32_t tag, *ctr;
            if (BITS == RADIX_BITS) {
                tag = p0 + p + 1;
                ctr = &ctl->tiles[p0 + p];
            } else {
                tag = MAX_PASSES + 1 + wpass;
                ctr = &ctl->wtiles[wpass];
                wpass++;
            }
            pass<K, ITEMS, BITS>(grid, at<K>(koff[src]), at<uint64_t>(voff[src]), at<K>(koff[dst]), at<uint64_t>(voff[dst]),
                                 n_ptr, n_max, BITS * p, dbase + (size_t)p * R, tag, ctr, tile_cap);
        }
        return (start + (int)np) & 1;
    }

    // LSD sort of (key, value) pairs that start in buffer `start` of 0/1; returns the buffer holding the
    // result. key_bits: the bits in use; p0: the first of the call's 8-bit passes for this stream; slot:
    // the stream's histogram region for other digit widths.
    template <class K>
    int sort(size_t koff[2], size_t voff[2], const uint32_t *n_ptr, uint64_t n_max, uint32_t key_bits, uint32_t p0,
             int start, uint32_t tile_cap, uint32_t slot) {
        const bool small = L.sort_items == 8;
        switch (L.radix_bits) {
            case 6:
                return small ? sort_w<K, 8, 6>(koff, voff, n_ptr, n_max, key_bits, p0, start, tile_cap, slot)
                             : sort_w<K, 16, 6>(koff, voff, n_ptr, n_max, key_bits, p0, start, tile_cap, slot);
            case 11:
                return small ? sort_w<K, 8, 11>(koff, voff, n_ptr, n_max, key_bits, p0, start, tile_cap, slot)
                             : sort_w<K, 16, 11>(koff, voff, n_ptr, n_max, key_bits, p0, start, tile_cap, slot);
            default:
                return small ? sort_w<K, 8, 8>(koff, voff, n_ptr, n_max, key_bits, p0, start, tile_cap, slot)
                             : sort_w<K, 16, 8>(koff, voff, n_ptr, n_max, key_bits, p0, start, tile_cap, slot);
        }
    }

    int grid_for(uint64_t items, uint64_t per_cta, uint64_t max_per_sm) const {
        return (int)std::max<uint64_t>(1, std::min<uint64_t>((items + per_cta - 1) / per_cta, (uint64_t)ctx->sms * max_per_sm));
    }
};

// Descriptors reach the device through kernel parameters (no host staging buffer, so a captured
// launch sequence carries them). The parameter block is read in place (__grid_constant__: no
// per-thread copy of it), one 4-byte word per thread.
constexpr int kDescChunk = 180;
constexpr int kDescWords = (int)(sizeof(TraceDesc) / 4);
static_assert(sizeof(TraceDesc) % 4 == 0, "descriptor words");
struct DescChunk {
    uint32_t w[kDescChunk * kDescWords];
};
static_assert(sizeof(DescChunk) + 16 < 32000, "descriptor chunk must fit the kernel parameter space");
constexpr int kDescThreads = 256;

__global__ void k_set_desc(uint32_t *dst, const __grid_constant__ DescChunk chunk, uint32_t words) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
        dst[i] = chunk.w[i];
}

// upload descriptors [0, T) to td on `st`; returns the launches issued
uint32_t upload_descs(TraceDesc *td, const std::vector<TraceDesc> &h, uint32_t T, cudaStream_t st) {
    uint32_t launches = 0;
    for (uint32_t i = 0; i < T; i += kDescChunk) {
        DescChunk c;
        const uint32_t cnt = std::min<uint32_t>(kDescChunk, T - i);
        memcpy(c.w, h.data() + i, cnt * sizeof(TraceDesc));
        const uint32_t words = cnt * kDescWords;
        k_set_desc<<<(words + kDescThreads - 1) / kDescThreads, kDescThreads, 0, st>>>(
            reinterpret_cast<uint32_t *>(td + i), c, words);
        launches++;
    }
    return launches;
}

// schedule-rank sort input: key (trace, visit order), value = batch-wide record index
template <class KQ>
__global__ void k_rank_init(const TraceDesc *td, Layout L, KQ *keys, uint64_t *vals, uint32_t *hist) {
    __shared__ uint32_t sh[8 * RADIX];
    for (int i = threadIdx.x; i < 8 * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < L.n; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = find_trace(L.T, r, [&](uint32_t i) { return td[i].rec_off; });
        const uint32_t vo = td[t].events[r - td[t].rec_off].y;
        const uint64_t k = shl(t, 32) | vo;
        keys[r] = (KQ)k;
        vals[r] = r;
        for (uint32_t p = 0; p < L.np_q; p++) atomicAdd(&sh[p * RADIX + digit_of(k, p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)(L.np_q * RADIX); i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

template <class KQ>
__global__ void k_rank_scatter(const KQ *sorted_keys, const uint64_t *sorted_idx, uint64_t n, uint32_t *rank,
                               uint32_t *pos_to_vo, Ctl *ctl) {
    if (must_stop(ctl)) return;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (sorted_idx[i] < n) rank[sorted_idx[i]] = (uint32_t)i;
        pos_to_vo[i] = (uint32_t)sorted_keys[i];
    }
}

__global__ void k_set_count(unsigned int *dst, unsigned int v) { *dst = v; }

// Fill host descriptors for a batch (block, record and tile offsets; outputs).
void fill_descs(const simulee_trace *tr, const simulee_outputs *outs, uint8_t *const *reports, uint32_t T,
                std::vector<TraceDesc> &td) {
    td.resize(T);
    uint64_t rec = 0, tile = 0, sig = 0;
    uint32_t blk = 0;
    for (uint32_t i = 0; i < T; i++) {
        TraceDesc &d = td[i];
        memset(&d, 0, sizeof d);
        d.events = (const uint4 *)tr[i].events;
        d.counts = tr[i].barrier_counts;
        d.n = tr[i].n_events;
        d.rec_off = rec;
        d.tile_off = tile;
        d.block_off = blk;
        d.nb = tr[i].n_blocks;
        d.bt = tr[i].block_threads;
        d.su = tr[i].shared_units;
        d.gu = tr[i].global_units;
        d.maxb = tr[i].max_barriers;
        d.flags = tr[i].flags;
        d.sig_off = sig;
        sig += tr[i].global_units;
        d.stmt = (tr[i].flags & SIMULEE_FLAG_WARP_AWARE) ? tr[i].stmt : nullptr;
        d.races = (uint8_t *)outs[i].races;
        d.races_cap = outs[i].races_cap;
        d.divs = (uint8_t *)outs[i].divergence;
        d.divs_cap = outs[i].divergence_cap;
        d.reds = (uint8_t *)outs[i].redundant;
        d.reds_cap = outs[i].redundant_cap;
        d.grid = outs[i].grid_redundant;
        d.grid_cap = outs[i].grid_redundant_cap;
        d.report = reports[i];
        rec += d.n;
        tile += (d.n + IN_TILE - 1) / IN_TILE;
        blk += d.nb;
    }
}

// the inter-block filter, instantiated for the key width and for the signature table's indexing
// (several traces in one direct table read each trace's offset; one trace or a hashed table does not)
void launch_x_filter(Run &R, const size_t xk[2], const size_t xv[2], uint32_t *sig, const TraceDesc *td,
                     uint32_t *hist) {
    const Layout &L = R.L;
    const int gf = R.grid_for(L.x_cap, XF_TILE, L.wide_x ? 2 : 3);   // resident CTAs per SM
    const bool offs = L.sig_direct && L.T > 1;
#define SIM_XF(KX, OFFS)                                                                                            \
    k_x_filter<KX, OFFS><<<gf, XF_THREADS, 0, R.st>>>(R.at<KX>(xk[0]), R.at<uint64_t>(xv[0]), R.at<KX>(xk[1]),        \
                                                   R.at<uint64_t>(xv[1]), sig, td, L, R.ctl, hist)
    if (L.wide_x) {
        if (offs) SIM_XF(uint64_t, true);
        else SIM_XF(uint64_t, false);
    } else {
        if (offs) SIM_XF(uint32_t, true);
        else SIM_XF(uint32_t, false);
    }
#undef SIM_XF
}

simulee_status issue_check(simulee_ctx *ctx, const simulee_trace *traces, uint32_t T, const simulee_outputs *outs,
                           uint8_t *const *reports, Want want, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !traces || !outs || !reports || !ws || T == 0) return SIMULEE_EINVAL;
    for (uint32_t i = 0; i < T; i++) {
        const simulee_status s = check_trace_args(&traces[i]);
        if (s != SIMULEE_OK) return s;
        const simulee_outputs &o = outs[i];
        if ((o.races_cap && !o.races) || (o.divergence_cap && !o.divergence) || (o.redundant_cap && !o.redundant) ||
            (o.grid_redundant_cap && !o.grid_redundant) || !reports[i])
            return SIMULEE_EINVAL;
    }
    if (((uintptr_t)ws & 255u) != 0) return SIMULEE_EINVAL;
    Run R;
    R.ctx = ctx;
    simulee_status s =
        make_layout(traces, T, ctx->sms, ctx->opt, R.L, Sizing::FIT, ctx->opt.path == SIMULEE_PATH_SORT, ws_bytes);
    if (s != SIMULEE_OK) return s;
    if (ws_bytes < R.L.total) return SIMULEE_ENOMEM;
    std::vector<TraceDesc> hdesc;
    fill_descs(traces, outs, reports, T, hdesc);
    bool any_hash = false;
    const bool route_any = want.races || want.red;
    for (uint32_t i = 0; i < T; i++) {
        TraceDesc &d = hdesc[i];
        d.hash_ok = (route_any && ctx->opt.path != SIMULEE_PATH_SORT &&
                     !(d.flags & (SIMULEE_FLAG_UNSORTED | SIMULEE_FLAG_WARP_AWARE | SIMULEE_FLAG_PAPER_ORDER)) &&
                     d.su < 0x7FFFFFFFu && d.gu < 0x7FFFFFFFu && d.n > 0) ? 1u : 0u;
        any_hash |= d.hash_ok != 0;
    }
    // hash-path CTA shapes: blocks of at most 256 threads go to two 512-thread CTAs per SM with
    // 4096-entry tables when there are at least two such blocks per SM (their runs hold fewer distinct
    // units than that table; one CTA's barriers overlap the other's work), the others to one
    // 768-thread CTA per SM with 8192-entry tables. The block list holds the first group, then the
    // second; each group is one launch.
    uint32_t nb_small = 0, nb_large = 0;
    for (uint32_t i = 0; i < T; i++)
        if (hdesc[i].hash_ok) (hdesc[i].bt <= 256 ? nb_small : nb_large) += hdesc[i].nb;
    bool split_small;
    if (ctx->opt.hash_shape == 1) split_small = false;
    else if (ctx->opt.hash_shape == 2) split_small = true;
    else split_small = nb_small >= 2u * (uint32_t)ctx->sms;
    // with a forced shape every block goes to its group
    const bool all_one = ctx->opt.hash_shape != 0 || !split_small;
    uint32_t n_first = 0, n_second = 0;
    {
        uint32_t o_first = 0, o_second = 0;
        for (uint32_t i = 0; i < T; i++) {
            TraceDesc &d = hdesc[i];
            if (!d.hash_ok) continue;
            const bool first = all_one || d.bt <= 256;
            if (first) { d.hlist = o_first; o_first += d.nb; }
            else { d.hlist = o_second; o_second += d.nb; }
        }
        n_first = o_first;
        n_second = o_second;
        for (uint32_t i = 0; i < T; i++)
            if (hdesc[i].hash_ok && !(all_one || hdesc[i].bt <= 256)) hdesc[i].hlist += n_first;
    }
    // the first group's shape: small when split (or forced small), else large; the second is large
    const bool first_small = all_one ? (ctx->opt.hash_shape == 2 || (ctx->opt.hash_shape == 0 && split_small))
                                     : true;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    if (!ctx->attrs_set) {
        set_sort_attr<uint32_t>();
        set_sort_attr<uint64_t>();
        set_reduce_attr<uint32_t, false>();
        set_reduce_attr<uint64_t, false>();
        set_reduce_attr<uint32_t, true>();
        set_reduce_attr<uint64_t, true>();
        set_hash_attr<uint32_t, HbLarge>();
        set_hash_attr<uint64_t, HbLarge>();
        set_hash_attr<uint32_t, HbSmall>();
        set_hash_attr<uint64_t, HbSmall>();
        set_hash_attr<uint32_t, HbHalf>();
        set_hash_attr<uint64_t, HbHalf>();
        set_hash_attr<uint32_t, HbQuarter>();
        set_hash_attr<uint64_t, HbQuarter>();
        ctx->attrs_set = true;
    }
    R.st = (cudaStream_t)stream;
    R.ws = (uint8_t *)ws;
    R.ctl = R.at<Ctl>(R.L.off_ctl);
    R.wait_ns = (uint64_t)(ctx->opt.wait_limit_us ? ctx->opt.wait_limit_us : 1000000u) * 1000ull;
    R.withhold = ctx->opt.test_withhold;
    const Layout &L = R.L;
    cudaStream_t st = R.st;
    TraceDesc *td = R.at<TraceDesc>(L.off_td);
    TState *ts = R.at<TState>(L.off_ts);
    uint32_t *tob = R.at<uint32_t>(L.off_tob);
    uint32_t *hist = R.at<uint32_t>(L.off_hist);

    // 1. zero control state, upload descriptors
    R.mark(SIMULEE_STAGE_INGEST, 0);
    cudaMemsetAsync(R.ws, 0, L.zero_end, st);
    cudaMemsetAsync(R.ws + L.off_status, 0, (size_t)L.status_tiles * status_digits(L) * 8, st);
    cudaMemsetAsync(R.ws + L.off_rgready, 0, (size_t)L.rg_tiles * 4, st);
    uint32_t *binel = R.at<uint32_t>(L.off_binel);
    uint32_t *spill = R.at<uint32_t>(L.off_spill);
    uint32_t *tflag = R.at<uint32_t>(L.off_tflag);
    uint32_t *fbt = R.at<uint32_t>(L.off_fbt);
    uint32_t *sig = L.sig_slots ? R.at<uint32_t>(L.off_sig) : nullptr;
    if (sig && (want.races || want.red)) cudaMemsetAsync(sig, 0, L.sig_slots * 4, st);
    R.launches += upload_descs(td, hdesc, T, st);
    k_block_trace<<<R.grid_for(L.NB, 256, 8), 256, 0, st>>>(td, L, tob);
    // 2. barrier counts
    k_block_stats<<<R.grid_for(L.NB, 8, 16), 256, 0, st>>>(td, tob, L, R.at<uint4>(L.off_stats), ts);
    R.launches += 2;

    const bool route = want.races || want.red;
    const bool sorting = L.n > 0 && route;
    bool any_sort = false;   // a trace on the sort path from the start
    for (uint32_t i = 0; i < T; i++) any_sort |= hdesc[i].hash_ok == 0 && hdesc[i].n > 0;
    uint32_t *rank = nullptr, *pos_to_vo = nullptr;
    if (L.any_unsorted) {
        rank = R.at<uint32_t>(L.off_rank);
        pos_to_vo = R.at<uint32_t>(L.off_p2v);
    }
    RaceStage rs;
    rs.keys = R.at<uint64_t>(L.off_rk[0]);
    rs.idx = R.at<uint64_t>(L.off_rv[0]);
    rs.pay = R.at<uint4>(L.off_rp);
    rs.cap = L.race_cap;
    rs.pos_to_vo = pos_to_vo;
    rs.n_pos = L.n;
    rs.ts = ts;
    rs.td = td;
    uint32_t *nonred = R.at<uint32_t>(L.off_nonred);
    if (L.n > 0) {
        // 3. unsorted traces: schedule rank of each record = position in (trace, visit order, index) order
        if (L.any_unsorted) {
            size_t qk[2] = {L.off_rk[0], L.off_rk[1]}, qv[2] = {L.off_rv[0], L.off_rv[1]};
            const int g = R.grid_for(L.n, 256, 8);
            uint32_t *hq = hist + (size_t)L.p0_q * RADIX, *dq = R.at<uint32_t>(L.off_dbase) + (size_t)L.p0_q * RADIX;
            if (L.wide_q) k_rank_init<uint64_t><<<g, 256, 0, st>>>(td, L, R.at<uint64_t>(qk[0]), R.at<uint64_t>(qv[0]), hq);
            else k_rank_init<uint32_t><<<g, 256, 0, st>>>(td, L, R.at<uint32_t>(qk[0]), R.at<uint64_t>(qv[0]), hq);
            k_digit_bases<<<L.np_q, RADIX, 0, st>>>(hq, dq, R.ctl);
            k_set_count<<<1, 1, 0, st>>>(&R.ctl->n_q, (unsigned int)L.n);
            R.launches += 3;
            const int b = L.wide_q ? R.sort<uint64_t>(qk, qv, &R.ctl->n_q, L.n, L.bits_q, L.p0_q, 0, 0, 4)
                                   : R.sort<uint32_t>(qk, qv, &R.ctl->n_q, L.n, L.bits_q, L.p0_q, 0, 0, 4);
            if (L.wide_q)
                k_rank_scatter<uint64_t><<<g, 256, 0, st>>>(R.at<uint64_t>(qk[b]), R.at<uint64_t>(qv[b]), L.n, rank,
                                                            pos_to_vo, R.ctl);
            else
                k_rank_scatter<uint32_t><<<g, 256, 0, st>>>(R.at<uint32_t>(qk[b]), R.at<uint64_t>(qv[b]), L.n, rank,
                                                            pos_to_vo, R.ctl);
            R.launches++;
        }

        // 4. ingest: validation-only read, or the first read of sort-path traces
        const int gi = R.grid_for(L.ntiles_in, 1, ctx->opt.ingest_ctas_per_sm ? ctx->opt.ingest_ctas_per_sm : 2u);
#define SIM_INGEST(KS, KG, KX, MODE)                                                                                \
    do {                                                                                                            \
        if (!attr_done(ctx, k_ingest<KS, KG, KX, MODE>))                                                            \
            cudaFuncSetAttribute(k_ingest<KS, KG, KX, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                 (int)ingest_smem());                                                               \
        k_ingest<KS, KG, KX, MODE><<<gi, IN_THREADS, ingest_smem(), st>>>(                                          \
            td, rank, L, ts, R.ctl, R.at<KS>(L.off_sk[0]), R.at<uint64_t>(L.off_sv[0]), R.at<KG>(L.off_gk[0]),      \
            R.at<uint64_t>(L.off_gv[0]), R.at<KX>(L.off_xk[0]), R.at<uint64_t>(L.off_xv[0]), hist, binel, spill,    \
            fbt, sig, R.wait_ns);                                                                                   \
    } while (0)
#define SIM_INGEST_W(MODE)                                                                                          \
    do {                                                                                                            \
        const int wmask = (L.wide_s ? 1 : 0) | (L.wide_g ? 2 : 0) | (L.wide_x ? 4 : 0);                             \
        if (wmask == 0) SIM_INGEST(uint32_t, uint32_t, uint32_t, MODE);                                              \
        else if (wmask == 1) SIM_INGEST(uint64_t, uint32_t, uint32_t, MODE);                                         \
        else if (wmask == 2) SIM_INGEST(uint32_t, uint64_t, uint32_t, MODE);                                         \
        else if (wmask == 3) SIM_INGEST(uint64_t, uint64_t, uint32_t, MODE);                                         \
        else if (wmask == 4) SIM_INGEST(uint32_t, uint32_t, uint64_t, MODE);                                         \
        else if (wmask == 5) SIM_INGEST(uint64_t, uint32_t, uint64_t, MODE);                                         \
        else if (wmask == 6) SIM_INGEST(uint32_t, uint64_t, uint64_t, MODE);                                         \
        else SIM_INGEST(uint64_t, uint64_t, uint64_t, MODE);                                                         \
        R.launches++;                                                                                               \
    } while (0)
        if (!route) {
            SIM_INGEST(uint32_t, uint32_t, uint32_t, IN_VALIDATE);
            R.launches++;
        } else if (any_sort) {
            SIM_INGEST_W(IN_FIRST);
        }
        R.mark(SIMULEE_STAGE_INGEST, 1);

        // 5. hash-path traces: one read of each block's records (validation, inter-block stream,
        //    intra-block checks), then the fallback read of what the hash path left to the sort path
        R.mark(SIMULEE_STAGE_HASH, 0);
        if (route && any_hash) {
            uint32_t *bstart = R.at<uint32_t>(L.off_bstart), *blist = R.at<uint32_t>(L.off_blist);
            uint32_t *bbins = R.at<uint32_t>(L.off_bbins), *gbeg = R.ctl->hb_gbeg;
            uint8_t *bgroup = R.at<uint8_t>(L.off_bgroup);
            // thread groups inside the smaller shape's CTAs for blocks with short runs
            const uint32_t groups_on = first_small && ctx->opt.hash_groups != 1 ? 1u : 0u;
            // list entries below small_end are blocks of the smaller shape, the rest of the larger
            const uint32_t small_end = first_small ? n_first : 0u, n_listed = n_first + n_second;
            // block ranges, launch group and size of each block, then each group's list with its
            // largest blocks first
            k_block_ranges<<<R.grid_for(L.NB, 8, 16), 256, 0, st>>>(td, tob, L, small_end, groups_on, bstart, bgroup,
                                                                    bbins);
            k_block_order<<<R.grid_for(L.NB, 256, 4), 256, 0, st>>>(td, tob, bstart, bgroup, L, bbins,
                                                                    bbins + HB_LGROUPS * HB_BINS, gbeg, blist);
            R.launches += 2;
#define SIM_HASH2(KX, SH, HOT, CNT, Q)                                                                               \
    k_hash_blocks<KX, SH, HOT><<<std::max(1, std::min<int>(ctx->sms * SH::ctas_per_sm,                              \
                                                           (int)(((CNT) + SH::groups - 1) / SH::groups))),           \
                                 SH::threads, hash_blocks_smem<SH>(), st>>>(                                         \
        td, tob, bstart, blist, gbeg, Q, R.at<uint4>(L.off_stats), &R.ctl->hb_next[Q], L, ts, R.ctl, nonred, binel,  \
        spill, tflag,                                                                                               \
        R.at<KX>(L.off_xk[0]), R.at<uint64_t>(L.off_xv[0]), sig, rs)
#define SIM_HASH(KX, SH, CNT, Q)                                                                                    \
    do {                                                                                                            \
        if (ctx->opt.hot_unit_marks == 2) SIM_HASH2(KX, SH, false, CNT, Q);                                         \
        else SIM_HASH2(KX, SH, true, CNT, Q);                                                                       \
    } while (0)
#define SIM_HASH_Q(KX, Q, CNT)                                                                                      \
    do {                                                                                                            \
        if ((Q) == HB_LG_QUARTER) SIM_HASH(KX, HbQuarter, CNT, Q);                                                  \
        else if ((Q) == HB_LG_HALF) SIM_HASH(KX, HbHalf, CNT, Q);                                                   \
        else if ((Q) == HB_LG_SMALL) SIM_HASH(KX, HbSmall, CNT, Q);                                                 \
        else SIM_HASH(KX, HbLarge, CNT, Q);                                                                         \
    } while (0)
            // launch groups in list order; the smaller class (small_end blocks) is split on the device
            // between the thread-group shapes and whole smaller CTAs, so each of those launches is
            // sized for the whole class and its CTAs read the group's true count
            for (int q = 0; q < HB_LGROUPS; q++) {
                const bool small_class = q != HB_LG_LARGE;
                const uint32_t cnt = small_class ? small_end : n_listed - small_end;
                if (cnt == 0) continue;
                if (small_class && !groups_on && q != HB_LG_SMALL) continue;
                if (L.wide_x) SIM_HASH_Q(uint64_t, q, cnt);
                else SIM_HASH_Q(uint32_t, q, cnt);
                R.launches++;
            }
#undef SIM_HASH_Q
#undef SIM_HASH
#undef SIM_HASH2
            R.mark(SIMULEE_STAGE_HASH, 1);
            R.mark(SIMULEE_STAGE_FALLBACK, 0);
            k_fallback_tiles<<<R.grid_for(L.ntiles_in, 256, 8), 256, 0, st>>>(td, L, ts, binel, tflag, R.ctl, fbt);
            R.launches++;
            SIM_INGEST_W(IN_FALLBACK);
            R.mark(SIMULEE_STAGE_FALLBACK, 1);
        } else {
            R.mark(SIMULEE_STAGE_HASH, 1);
            R.mark(SIMULEE_STAGE_FALLBACK, 0);
            R.mark(SIMULEE_STAGE_FALLBACK, 1);
        }
#undef SIM_INGEST_W
#undef SIM_INGEST
    } else {
        R.mark(SIMULEE_STAGE_INGEST, 1);
        R.mark(SIMULEE_STAGE_HASH, 0);
        R.mark(SIMULEE_STAGE_HASH, 1);
        R.mark(SIMULEE_STAGE_FALLBACK, 0);
        R.mark(SIMULEE_STAGE_FALLBACK, 1);
    }

    // 6. sort the three streams
    R.mark(SIMULEE_STAGE_SORT, 0);
    int bs = 0, bg = 0, bx = 0;
    if (sorting) {
        size_t sk[2] = {L.off_sk[0], L.off_sk[1]}, sv[2] = {L.off_sv[0], L.off_sv[1]};
        size_t gk[2] = {L.off_gk[0], L.off_gk[1]}, gv[2] = {L.off_gv[0], L.off_gv[1]};
        size_t xk[2] = {L.off_xk[0], L.off_xk[1]}, xv[2] = {L.off_xv[0], L.off_xv[1]};
        if (L.any_paper) {
            // the intra-block streams first (their digit bases come from the record reads); the inter-block
            // elements of traces with the paper's visit-order counters come from the sorted global stream
            uint32_t *dbase = R.at<uint32_t>(L.off_dbase);
            if (L.p0_x > 0) {
                k_digit_bases<<<L.p0_x, RADIX, 0, st>>>(hist, dbase, R.ctl);
                R.launches++;
            }
            bs = L.wide_s ? R.sort<uint64_t>(sk, sv, &R.ctl->n_s, L.cap_s, L.bits_s, L.p0_s, 0, 0, 0)
                          : R.sort<uint32_t>(sk, sv, &R.ctl->n_s, L.cap_s, L.bits_s, L.p0_s, 0, 0, 0);
            bg = L.wide_g ? R.sort<uint64_t>(gk, gv, &R.ctl->n_g, L.cap_s, L.bits_g, L.p0_g, 0, 0, 1)
                          : R.sort<uint32_t>(gk, gv, &R.ctl->n_g, L.cap_s, L.bits_g, L.p0_g, 0, 0, 1);
            const int gp = R.grid_for(L.n, PX_TILE, 4);
            unsigned long long *stw = R.at<unsigned long long>(L.off_status);
#define SIM_PX(KG, KX)                                                                                            \
    k_paper_x<KG, KX><<<gp, PX_THREADS, 0, st>>>(R.at<KG>(gk[bg]), R.at<uint64_t>(gv[bg]), &R.ctl->n_g, L, td, tob, \
                                                stw, R.ctl, R.at<KX>(xk[0]), R.at<uint64_t>(xv[0]), R.wait_ns)
            if (L.wide_g) {
                if (L.wide_x) SIM_PX(uint64_t, uint64_t);
                else SIM_PX(uint64_t, uint32_t);
            } else {
                if (L.wide_x) SIM_PX(uint32_t, uint64_t);
                else SIM_PX(uint32_t, uint32_t);
            }
#undef SIM_PX
            R.launches++;
            if (L.sig_slots) {
                launch_x_filter(R, xk, xv, sig, td, hist);
                R.launches++;
            }
            if (L.np_x > 0) {
                k_digit_bases<<<L.np_x, RADIX, 0, st>>>(hist + (size_t)L.p0_x * RADIX, dbase + (size_t)L.p0_x * RADIX,
                                                        R.ctl);
                R.launches++;
            }
            bx = L.wide_x ? R.sort<uint64_t>(xk, xv, &R.ctl->n_xf, L.cap_x1, L.bits_x, L.p0_x, 1, 0, 2)
                          : R.sort<uint32_t>(xk, xv, &R.ctl->n_xf, L.cap_x1, L.bits_x, L.p0_x, 1, 0, 2);
        } else {
        // inter-block records of units touched by one block only are dropped before sorting;
        // the filter also builds the inter stream's digit histograms
        if (L.sig_slots) {
            launch_x_filter(R, xk, xv, sig, td, hist);
            R.launches++;
        }
        if (L.p0_r > 0) {
            k_digit_bases<<<L.p0_r, RADIX, 0, st>>>(hist, R.at<uint32_t>(L.off_dbase), R.ctl);
            R.launches++;
        }
        bs = L.wide_s ? R.sort<uint64_t>(sk, sv, &R.ctl->n_s, L.cap_s, L.bits_s, L.p0_s, 0, 0, 0)
                      : R.sort<uint32_t>(sk, sv, &R.ctl->n_s, L.cap_s, L.bits_s, L.p0_s, 0, 0, 0);
        bg = L.wide_g ? R.sort<uint64_t>(gk, gv, &R.ctl->n_g, L.cap_s, L.bits_g, L.p0_g, 0, 0, 1)
                      : R.sort<uint32_t>(gk, gv, &R.ctl->n_g, L.cap_s, L.bits_g, L.p0_g, 0, 0, 1);
        bx = L.wide_x ? R.sort<uint64_t>(xk, xv, &R.ctl->n_xf, L.cap_x1, L.bits_x, L.p0_x, 1, 0, 2)
                      : R.sort<uint32_t>(xk, xv, &R.ctl->n_xf, L.cap_x1, L.bits_x, L.p0_x, 1, 0, 2);
        }
    }
    R.mark(SIMULEE_STAGE_SORT, 1);

    // 7. segmented reductions
    R.mark(SIMULEE_STAGE_REDUCE, 0);
    if (sorting) {
        const int gr = R.grid_for(L.n, RG_TILE, ctx->opt.reduce_ctas_per_sm ? ctx->opt.reduce_ctas_per_sm : 3u);
        // the three launches share the published tile summaries; their ready words carry tags 1, 2, 3
#define SIM_REDUCE(K, INTER, KOFF, VOFF, NPTR, NMAX, SPACE, BU, SLOT)                                                 \
    k_reduce_groups<K, INTER><<<gr, RG_THREADS, reduce_groups_smem<K, INTER>(), st>>>(                                \
        R.at<K>(KOFF), R.at<uint64_t>(VOFF), NPTR, NMAX, L, td, tob, SPACE, BU, R.ctl, nonred, rs,                     \
        R.at<RgTile>(L.off_rgpub), R.at<uint32_t>(L.off_rgready), SLOT + 1u, &R.ctl->rg_tiles[SLOT], R.wait_ns)
        if (L.wide_s) SIM_REDUCE(uint64_t, false, L.off_sk[bs], L.off_sv[bs], &R.ctl->n_s, L.cap_s, 0u, L.bus, 0u);
        else SIM_REDUCE(uint32_t, false, L.off_sk[bs], L.off_sv[bs], &R.ctl->n_s, L.cap_s, 0u, L.bus, 0u);
        if (L.wide_g) SIM_REDUCE(uint64_t, false, L.off_gk[bg], L.off_gv[bg], &R.ctl->n_g, L.cap_s, 1u, L.bug, 1u);
        else SIM_REDUCE(uint32_t, false, L.off_gk[bg], L.off_gv[bg], &R.ctl->n_g, L.cap_s, 1u, L.bug, 1u);
        if (L.wide_x) SIM_REDUCE(uint64_t, true, L.off_xk[bx], L.off_xv[bx], &R.ctl->n_xf, L.cap_x1, 1u, L.bug, 2u);
        else SIM_REDUCE(uint32_t, true, L.off_xk[bx], L.off_xv[bx], &R.ctl->n_xf, L.cap_x1, 1u, L.bug, 2u);
#undef SIM_REDUCE
        R.launches += 3;
    }
    R.mark(SIMULEE_STAGE_REDUCE, 1);

    // 8. races in canonical order, split per trace
    R.mark(SIMULEE_STAGE_RACES, 0);
    if (sorting && want.races) {
        k_race_filter<<<R.grid_for(L.race_cap, 256, 4), 256, 0, st>>>(
            rs.keys, rs.idx, R.at<uint64_t>(L.off_rk[1]), R.at<uint64_t>(L.off_rv[1]), L, binel, ts, R.ctl, hist);
        k_digit_bases<<<L.np_r, RADIX, 0, st>>>(hist + (size_t)L.p0_r * RADIX,
                                                R.at<uint32_t>(L.off_dbase) + (size_t)L.p0_r * RADIX, R.ctl);
        R.launches += 2;
        size_t rk[2] = {L.off_rk[0], L.off_rk[1]}, rv[2] = {L.off_rv[0], L.off_rv[1]};
        // race records are few next to the record streams: at most 128 tiles keeps their look-back short
        const int br = R.sort<uint64_t>(rk, rv, &R.ctl->n_rf, L.race_cap, L.bits_r, L.p0_r, 1, 128u, 3);
        const int gw = R.grid_for(L.race_cap, 256, 8);
        if (T > 1) {   // one trace: its races start at 0 (the per-trace state is zeroed)
            k_race_starts<<<gw, 256, 0, st>>>(R.at<uint64_t>(rk[br]), L, R.ctl, ts);
            R.launches++;
        }
        k_write_races<<<gw, 256, 0, st>>>(R.at<uint64_t>(rk[br]), R.at<uint64_t>(rv[br]), rs.pay, L, td, ts, R.ctl);
        R.launches++;
    }
    R.mark(SIMULEE_STAGE_RACES, 1);

    // 9. per-block outputs and reports
    R.mark(SIMULEE_STAGE_BLOCKS, 0);
    uint32_t *ofs_div = R.at<uint32_t>(L.off_ofs_div), *ofs_red = R.at<uint32_t>(L.off_ofs_red);
    const int gb = R.grid_for(L.NB, 256, 8);
    k_block_counts<<<gb, 256, 0, st>>>(R.at<uint4>(L.off_stats), nonred, L, R.at<uint32_t>(L.off_cnt_div),
                                       R.at<uint32_t>(L.off_cnt_red));
    k_scan2<<<1, 1024, 0, st>>>(R.at<uint32_t>(L.off_cnt_div), R.at<uint32_t>(L.off_cnt_red), L.NB, ofs_div, ofs_red,
                                R.ctl);
    R.launches += 2;
    if (want.div || want.red) {
        k_block_write<<<gb, 256, 0, st>>>(R.at<uint4>(L.off_stats), nonred, L, td, tob, ts, ofs_div, ofs_red,
                                          want.div ? 1u : 0u, want.red ? 1u : 0u);
        R.launches++;
    }
    if (want.red) {
        k_grid_or<<<R.grid_for((uint64_t)L.NB * L.words, 256, 8), 256, 0, st>>>(
            R.at<uint4>(L.off_stats), nonred, tob, L, R.at<uint32_t>(L.off_gridnr), R.at<uint32_t>(L.off_gridhas));
        k_grid_list<<<T, 1024, 0, st>>>(R.at<uint32_t>(L.off_gridnr), R.at<uint32_t>(L.off_gridhas), L, td, ts);
        R.launches += 2;
    }
    ReportArgs ra;
    ra.want_races = want.races;
    ra.want_div = want.div;
    ra.want_red = want.red;
    k_report<<<R.grid_for(T, 256, 4), 256, 0, st>>>(td, ts, ofs_div, ofs_red, L, R.ctl, ra);
    R.launches++;
    R.mark(SIMULEE_STAGE_BLOCKS, 1);
    ctx->last_launches = R.launches;
    const cudaError_t e = cudaGetLastError();
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
}

// Every argument a check's launch sequence depends on, as bytes: two calls with equal keys issue the
// same kernels with the same parameters (the device data they read may differ).
std::vector<uint8_t> call_key(const simulee_ctx *ctx, const simulee_trace *traces, uint32_t T,
                              const simulee_outputs *outs, uint8_t *const *reports, Want want, void *ws,
                              size_t ws_bytes) {
    std::vector<uint8_t> k;
    auto put = [&k](const void *p, size_t n) {
        const uint8_t *b = (const uint8_t *)p;
        k.insert(k.end(), b, b + n);
    };
    put(&ctx->opt, sizeof ctx->opt);
    put(&T, sizeof T);
    const uint8_t w[3] = {want.races, want.div, want.red};
    put(w, 3);
    put(&ws, sizeof ws);
    put(&ws_bytes, sizeof ws_bytes);
    for (uint32_t i = 0; i < T; i++) {
        put(&traces[i], sizeof traces[i]);
        put(&outs[i], sizeof outs[i]);
        put(&reports[i], sizeof reports[i]);
    }
    return k;
}

// A check. A call whose arguments equal those of the call just before it on this context is issued
// as a CUDA graph: the second such call captures the launch sequence (on a private stream, without
// running it) and launches the graph on the caller's stream; later equal calls launch it again. The
// graph's kernels read the trace, write the outputs and use the workspace at run time, exactly as
// the direct launches do. Direct launches are used when graph replay is off in the options, when
// stage events are on, and when the caller's stream is itself being captured.
simulee_status run_check(simulee_ctx *ctx, const simulee_trace *traces, uint32_t T, const simulee_outputs *outs,
                         uint8_t *const *reports, Want want, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !traces || !outs || !reports || !ws || T == 0) return SIMULEE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    ctx->last_replayed = 0;
    if (ctx->opt.graph_replay == SIMULEE_GRAPH_OFF || ctx->stage_on || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return issue_check(ctx, traces, T, outs, reports, want, ws, ws_bytes, stream);
    std::vector<uint8_t> key = call_key(ctx, traces, T, outs, reports, want, ws, ws_bytes);
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    auto restore = [&]() {
        if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    };
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    if (ctx->graph_exec && key == ctx->graph_key) {
        const cudaError_t e = cudaGraphLaunch(ctx->graph_exec, st);
        ctx->last_launches = ctx->graph_launches;
        ctx->last_replayed = e == cudaSuccess ? 1u : 0u;
        restore();
        return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
    }
    if (key != ctx->seen_key) {   // first sighting: direct launches
        restore();
        const simulee_status s = issue_check(ctx, traces, T, outs, reports, want, ws, ws_bytes, stream);
        ctx->seen_key = s == SIMULEE_OK ? std::move(key) : std::vector<uint8_t>();
        return s;
    }
    // the same arguments twice in a row: capture, instantiate, launch
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        ctx->cap_stream = nullptr;
        restore();
        return issue_check(ctx, traces, T, outs, reports, want, ws, ws_bytes, stream);
    }
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        restore();
        return issue_check(ctx, traces, T, outs, reports, want, ws, ws_bytes, stream);
    }
    const simulee_status s = issue_check(ctx, traces, T, outs, reports, want, ws, ws_bytes, ctx->cap_stream);
    cudaSetDevice(ctx->device);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
    cudaGraphExec_t ex = nullptr;
    const bool ok = s == SIMULEE_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        if (ex) cudaGraphExecDestroy(ex);
        restore();
        if (s != SIMULEE_OK) return s;
        return issue_check(ctx, traces, T, outs, reports, want, ws, ws_bytes, stream);
    }
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = ex;
    ctx->graph_key = std::move(key);
    ctx->graph_launches = ctx->last_launches;
    const cudaError_t e = cudaGraphLaunch(ex, st);
    ctx->last_replayed = e == cudaSuccess ? 1u : 0u;
    restore();
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
}

// ---- fitness (Eq. 1) -------------------------------------------------------------------------
static_assert(sizeof(simulee_fitness) == FIT_OUT_BYTES, "simulee_fitness layout");
struct FitPlan {
    Layout L;       // the fields the validation kernels read (n, T, NB, ntiles_in, maxb)
    FitKeys fk;
    bool wide;
    uint64_t status_tiles;
    bool single;           // the single read applies (the bitmap of all traces' global units is small enough)
    uint32_t fb_ctas;      // CTAs of the single read, one table each
    uint64_t gbit_words;   // 32-bit words of the global-unit bitmap
    size_t off_ctl, off_ts, off_acc, off_hist, off_td, off_tob, off_stats, off_dbase, off_status, off_k[2];
    size_t off_fb, off_gbits, off_bstart, off_tabs;
    size_t zero_end, total;
};

// The single read's global-unit bitmap holds every trace's global units (one bit each) up to this many
// bits (1 GiB); a batch with more is counted from sorted keys.
constexpr uint64_t kFitMaxGlobalBits = 1ull << 33;

simulee_status fit_plan(const simulee_trace *tr, uint32_t T, int sms, FitPlan &P) {
    memset(&P, 0, sizeof P);
    if (!tr || T == 0 || T > kMaxTraces) return SIMULEE_EINVAL;
    uint64_t n = 0, nb = 0, tiles = 0, maxthreads = 0;
    uint32_t maxb = 0, maxnb = 0, units = 0;
    uint64_t gbits = 0;
    for (uint32_t i = 0; i < T; i++) {
        const simulee_status s = check_trace_args(&tr[i]);
        if (s != SIMULEE_OK) return s;
        gbits += tr[i].global_units;
        n += tr[i].n_events;
        nb += tr[i].n_blocks;
        tiles += (tr[i].n_events + IN_TILE - 1) / IN_TILE;
        maxb = std::max(maxb, tr[i].max_barriers);
        maxnb = std::max(maxnb, tr[i].n_blocks);
        units = std::max(units, std::max(tr[i].shared_units, tr[i].global_units));
        maxthreads = std::max<uint64_t>(maxthreads, (uint64_t)tr[i].n_blocks * tr[i].block_threads);
    }
    if (n >= (1ull << 31) || nb >= (1ull << 31)) return SIMULEE_EINVAL;
    Layout &L = P.L;
    L.n = n;
    L.T = T;
    L.NB = (uint32_t)nb;
    L.ntiles_in = tiles;
    L.maxb = maxb;
    FitKeys &f = P.fk;
    f.bg = bits_for(maxthreads);
    f.bu = bits_for(units);
    f.bbl = bits_for(maxnb);
    f.btr = bits_for(T);
    f.bits = f.bg + f.bu + f.bbl + 1 + f.btr;
    if (f.bits > 64) return SIMULEE_EINVAL;
    f.np = passes_for(f.bits);
    if (f.np > 8) return SIMULEE_EINVAL;
    P.wide = f.bits > 32;
    const uint64_t n1 = std::max<uint64_t>(n, 1);
    P.status_tiles = (n1 + OS_TILE - 1) / OS_TILE;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
    P.single = n > 0 && gbits <= kFitMaxGlobalBits;
    P.gbit_words = P.single ? (gbits + 31) / 32 : 0;
    P.fb_ctas = P.single ? (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(nb, (uint64_t)sms)) : 0;
    P.off_ctl = take(sizeof(Ctl));
    P.off_ts = take((size_t)T * sizeof(TState));
    P.off_hist = take((size_t)8 * RADIX * 4);
    P.off_fb = take((size_t)nb * 4);
    P.off_gbits = take((size_t)P.gbit_words * 4);
    P.zero_end = o;
    P.off_bstart = take((size_t)nb * 4);
    P.off_tabs = take((size_t)P.fb_ctas * FB_SLOTS * 8);
    P.off_acc = take((size_t)T * sizeof(FitAcc));
    P.off_td = take((size_t)T * sizeof(TraceDesc));
    P.off_tob = take((size_t)nb * 4);
    P.off_stats = take((size_t)nb * 16);
    P.off_dbase = take((size_t)8 * RADIX * 4);
    P.off_status = take((size_t)P.status_tiles * RADIX * 8);
    for (int i = 0; i < 2; i++) P.off_k[i] = take(n1 * (P.wide ? 8 : 4));
    P.total = o;
    return SIMULEE_OK;
}

simulee_status run_fitness(simulee_ctx *ctx, const simulee_trace *traces, uint32_t T, simulee_fitness *out, void *ws,
                           size_t ws_bytes, void *stream) {
    if (!ctx || !traces || !out || !ws || T == 0) return SIMULEE_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SIMULEE_EINVAL;
    FitPlan P;
    simulee_status s = fit_plan(traces, T, ctx->sms, P);
    if (s != SIMULEE_OK) return s;
    if (ws_bytes < P.total) return SIMULEE_ENOMEM;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    const Layout &L = P.L;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *w = (uint8_t *)ws;
    Ctl *ctl = reinterpret_cast<Ctl *>(w + P.off_ctl);
    TState *ts = reinterpret_cast<TState *>(w + P.off_ts);
    FitAcc *acc = reinterpret_cast<FitAcc *>(w + P.off_acc);
    TraceDesc *td = reinterpret_cast<TraceDesc *>(w + P.off_td);
    uint32_t *tob = reinterpret_cast<uint32_t *>(w + P.off_tob);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + P.off_hist);
    uint32_t *dbase = reinterpret_cast<uint32_t *>(w + P.off_dbase);
    const uint64_t wait_ns = (uint64_t)(ctx->opt.wait_limit_us ? ctx->opt.wait_limit_us : 1000000u) * 1000ull;
    uint32_t launches = 0;
    auto grid_for = [&](uint64_t items, uint64_t per_cta, uint64_t per_sm) {
        return (int)std::max<uint64_t>(1, std::min<uint64_t>((items + per_cta - 1) / per_cta, (uint64_t)ctx->sms * per_sm));
    };
    cudaMemsetAsync(w, 0, P.zero_end, st);
    cudaMemsetAsync(w + P.off_status, 0, (size_t)P.status_tiles * RADIX * 8, st);
    // descriptors: the check's, without outputs
    std::vector<simulee_outputs> no_out(T);
    memset(no_out.data(), 0, T * sizeof(simulee_outputs));
    std::vector<uint8_t *> no_rep(T, nullptr);
    std::vector<TraceDesc> hdesc;
    fill_descs(traces, no_out.data(), no_rep.data(), T, hdesc);
    // traces counted by the single read (sig_off: the bit of the trace's global unit 0 in the bitmap):
    // those with at least 1024 records per block on average; a 1024-thread CTA per block would idle on
    // smaller blocks, which the sort takes in bulk
    for (uint32_t i = 0; i < T; i++)
        hdesc[i].hash_ok = P.single && hdesc[i].n > 0 && hdesc[i].n >= 1024ull * hdesc[i].nb ? 1u : 0u;
    launches += upload_descs(td, hdesc, T, st);
    k_fit_init<<<grid_for(T, 256, 1), 256, 0, st>>>(td, acc, T);
    k_block_trace<<<grid_for(L.NB, 256, 8), 256, 0, st>>>(td, L, tob);
    k_block_stats<<<grid_for(L.NB, 8, 16), 256, 0, st>>>(td, tob, L, reinterpret_cast<uint4 *>(w + P.off_stats), ts);
    launches += 3;
    if (L.n > 0) {
        // validation: the check's record read, validation only
        if (!attr_done(ctx, k_ingest<uint32_t, uint32_t, uint32_t, IN_VALIDATE>))
            cudaFuncSetAttribute(k_ingest<uint32_t, uint32_t, uint32_t, IN_VALIDATE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ingest_smem());
        const int gi = grid_for(L.ntiles_in, 1, 2);
        k_ingest<uint32_t, uint32_t, uint32_t, IN_VALIDATE><<<gi, IN_THREADS, ingest_smem(), st>>>(
            td, nullptr, L, ts, ctl, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, hist, nullptr, nullptr,
            nullptr, nullptr, wait_ns);
        launches++;
        // the single read: block ranges, then one CTA per block with a table of its own
        uint32_t *fb = reinterpret_cast<uint32_t *>(w + P.off_fb);
        if (P.single) {
            uint32_t *bstart = reinterpret_cast<uint32_t *>(w + P.off_bstart);
            k_fit_ranges<<<grid_for(L.NB, 8, 16), 256, 0, st>>>(td, tob, L, bstart);
            k_fit_blocks<<<P.fb_ctas, FB_THREADS, 0, st>>>(
                td, tob, bstart, L, ts, &ctl->hb_next[0], reinterpret_cast<unsigned long long *>(w + P.off_tabs),
                reinterpret_cast<uint32_t *>(w + P.off_gbits), acc, fb);
            launches += 2;
        }
        // what the single read left (ctl->n_q records) through the radix sort
        const int gk = grid_for(L.ntiles_in, 1, 8);
        const int gs = grid_for(L.n, OS_TILE, 3);
#define SIM_FIT(K)                                                                                                 \
    do {                                                                                                           \
        if (!attr_done(ctx, k_onesweep<K>))                                                                        \
            cudaFuncSetAttribute(k_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem<K>()); \
        K *k0 = reinterpret_cast<K *>(w + P.off_k[0]), *k1 = reinterpret_cast<K *>(w + P.off_k[1]);                 \
        k_fit_keys<K><<<gk, FK_THREADS, 0, st>>>(td, L, P.fk, fb, k0, hist, acc, ctl);                            \
        k_digit_bases<<<P.fk.np, RADIX, 0, st>>>(hist, dbase, ctl);                                                \
        launches += 2;                                                                                             \
        K *bufs[2] = {k0, k1};                                                                                     \
        for (uint32_t p = 0; p < P.fk.np; p++) {                                                                   \
            k_onesweep<K><<<gs, OS_THREADS, onesweep_smem<K>(), st>>>(                                             \
                bufs[p & 1], nullptr, bufs[(p & 1) ^ 1], nullptr, &ctl->n_q, L.n, RADIX_BITS * p,                  \
                dbase + (size_t)p * RADIX, reinterpret_cast<unsigned long long *>(w + P.off_status), p + 1,        \
                &ctl->tiles[p], ctl, wait_ns, 0u, 0u);                                                             \
            launches++;                                                                                            \
        }                                                                                                          \
        k_fit_count<K><<<grid_for(L.n, 256, 8), 256, 0, st>>>(bufs[P.fk.np & 1], &ctl->n_q, P.fk, T, acc, ctl);    \
        launches++;                                                                                                \
    } while (0)
        if (P.wide) SIM_FIT(uint64_t);
        else SIM_FIT(uint32_t);
#undef SIM_FIT
    }
    k_fit_report<<<grid_for(T, 256, 1), 256, 0, st>>>(ts, acc, T, ctl, reinterpret_cast<uint8_t *>(out));
    launches++;
    ctx->last_launches = launches;
    const cudaError_t e = cudaGetLastError();
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
}

simulee_status launch_check(simulee_ctx *ctx, const simulee_trace *t, const simulee_outputs *out, Want want,
                            simulee_report *report, void *ws, size_t ws_bytes, void *stream) {
    if (!out || !report) return SIMULEE_EINVAL;
    uint8_t *rep = (uint8_t *)report;
    return run_check(ctx, t, 1, out, &rep, want, ws, ws_bytes, stream);
}

}  // namespace

extern "C" {

simulee_status simulee_create(simulee_ctx **ctx, int device, const simulee_options *opt) {
    if (!ctx) return SIMULEE_EINVAL;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SIMULEE_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SIMULEE_ECUDA;
    if (opt) {
        if (opt->sort_items != 0 && opt->sort_items != 8 && opt->sort_items != 16) return SIMULEE_EINVAL;
        if (opt->radix_bits != 0 && opt->radix_bits != 6 && opt->radix_bits != 8 && opt->radix_bits != 11)
            return SIMULEE_EINVAL;
        if (opt->hash_cap_eighths != 0 && (opt->hash_cap_eighths < 4 || opt->hash_cap_eighths > 7)) return SIMULEE_EINVAL;
        if (opt->hot_unit_marks > 2) return SIMULEE_EINVAL;
        if (opt->hash_groups > 1) return SIMULEE_EINVAL;
        if (opt->hash_pool_div != 0 && (opt->hash_pool_div < 3 || opt->hash_pool_div > 64)) return SIMULEE_EINVAL;
    }
    simulee_ctx *c = new (std::nothrow) simulee_ctx();
    if (!c) return SIMULEE_ENOMEM;
    c->device = device;
    c->sms = prop.multiProcessorCount;
    if (opt) c->opt = *opt;
    *ctx = c;
    return SIMULEE_OK;
}

simulee_status simulee_destroy(simulee_ctx *ctx) {
    if (!ctx) return SIMULEE_EINVAL;
    delete ctx;
    return SIMULEE_OK;
}

simulee_status simulee_workspace_size(simulee_ctx *ctx, const simulee_trace *trace, size_t *bytes) {
    if (!ctx || !trace || !bytes) return SIMULEE_EINVAL;
    Layout L;
    const simulee_status s = make_layout(trace, 1, ctx->sms, ctx->opt, L);
    if (s != SIMULEE_OK) return s;
    *bytes = L.total;
    return SIMULEE_OK;
}

simulee_status simulee_compact_workspace_size(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                              size_t *bytes) {
    if (!ctx || !traces || !bytes || n_traces == 0) return SIMULEE_EINVAL;
    Layout L;
    const simulee_status s =
        make_layout(traces, n_traces, ctx->sms, ctx->opt, L, Sizing::COMPACT, ctx->opt.path == SIMULEE_PATH_SORT);
    if (s != SIMULEE_OK) return s;
    *bytes = L.total;
    return SIMULEE_OK;
}

simulee_status simulee_check(simulee_ctx *ctx, const simulee_trace *trace, const simulee_outputs *out,
                             simulee_report *report, void *ws, size_t ws_bytes, void *stream) {
    return launch_check(ctx, trace, out, Want{true, true, true}, report, ws, ws_bytes, stream);
}

simulee_status simulee_check_races(simulee_ctx *ctx, const simulee_trace *trace, simulee_race *out, uint64_t cap,
                                   simulee_report *report, void *ws, size_t ws_bytes, void *stream) {
    simulee_outputs o;
    memset(&o, 0, sizeof o);
    o.races = out;
    o.races_cap = cap;
    return launch_check(ctx, trace, &o, Want{true, false, false}, report, ws, ws_bytes, stream);
}

simulee_status simulee_check_divergence(simulee_ctx *ctx, const simulee_trace *trace, simulee_divergence *out,
                                        uint64_t cap, simulee_report *report, void *ws, size_t ws_bytes,
                                        void *stream) {
    simulee_outputs o;
    memset(&o, 0, sizeof o);
    o.divergence = out;
    o.divergence_cap = cap;
    return launch_check(ctx, trace, &o, Want{false, true, false}, report, ws, ws_bytes, stream);
}

simulee_status simulee_check_redundant_barriers(simulee_ctx *ctx, const simulee_trace *trace, simulee_barrier *out,
                                                uint64_t cap, uint32_t *grid, uint64_t grid_cap,
                                                simulee_report *report, void *ws, size_t ws_bytes, void *stream) {
    simulee_outputs o;
    memset(&o, 0, sizeof o);
    o.redundant = out;
    o.redundant_cap = cap;
    o.grid_redundant = grid;
    o.grid_redundant_cap = grid_cap;
    return launch_check(ctx, trace, &o, Want{false, false, true}, report, ws, ws_bytes, stream);
}

simulee_status simulee_batch_workspace_size(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                            size_t *bytes) {
    if (!ctx || !traces || !bytes || n_traces == 0) return SIMULEE_EINVAL;
    Layout L;
    const simulee_status s = make_layout(traces, n_traces, ctx->sms, ctx->opt, L);
    if (s != SIMULEE_OK) return s;
    *bytes = L.total;
    return SIMULEE_OK;
}

simulee_status simulee_check_batch(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                   const simulee_outputs *outs, simulee_report *reports, void *ws, size_t ws_bytes,
                                   void *stream) {
    if (!reports || n_traces == 0 || n_traces > kMaxTraces) return SIMULEE_EINVAL;
    std::vector<uint8_t *> reps(n_traces);
    for (uint32_t i = 0; i < n_traces; i++) reps[i] = (uint8_t *)(reports + i);
    return run_check(ctx, traces, n_traces, outs, reps.data(), Want{true, true, true}, ws, ws_bytes, stream);
}

simulee_status simulee_fitness_workspace_size(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                              size_t *bytes) {
    if (!ctx || !traces || !bytes) return SIMULEE_EINVAL;
    FitPlan P;
    const simulee_status s = fit_plan(traces, n_traces, ctx->sms, P);
    if (s != SIMULEE_OK) return s;
    *bytes = P.total;
    return SIMULEE_OK;
}

simulee_status simulee_fitness_batch(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                     simulee_fitness *out, void *ws, size_t ws_bytes, void *stream) {
    return run_fitness(ctx, traces, n_traces, out, ws, ws_bytes, stream);
}

simulee_status simulee_model_traces(simulee_ctx *ctx, const simulee_model *models, uint32_t n_models,
                                    simulee_event *events, uint64_t n_events, uint32_t *counts, uint64_t n_counts,
                                    void *stream) {
    if (!ctx || !models || n_models == 0 || (n_events && !events) || (n_counts && !counts)) return SIMULEE_EINVAL;
    if (((uintptr_t)events & 15u) != 0) return SIMULEE_EINVAL;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    const uint64_t work = std::max(n_events, n_counts);
    const int g = (int)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)ctx->sms * 8));
    k_model_traces<<<g, 256, 0, (cudaStream_t)stream>>>(models, n_models, n_events, reinterpret_cast<uint4 *>(events),
                                                       n_counts, counts);
    ctx->last_launches = 1;
    const cudaError_t e = cudaGetLastError();
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
}

uint32_t simulee_last_launches(const simulee_ctx *ctx) { return ctx ? ctx->last_launches : 0u; }

uint32_t simulee_last_replayed(const simulee_ctx *ctx) { return ctx ? ctx->last_replayed : 0u; }

simulee_status simulee_stream_sizes(simulee_ctx *ctx, const void *ws, uint32_t *dev_out, void *stream) {
    if (!ctx || !ws || !dev_out) return SIMULEE_EINVAL;
    static_assert(offsetof(Ctl, n_x) == offsetof(Ctl, n_s) + 16, "stream counters are contiguous");
    const cudaError_t e = cudaMemcpyAsync(dev_out, (const uint8_t *)ws + offsetof(Ctl, n_s), 20,
                                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
}

simulee_status simulee_hash_groups(simulee_ctx *ctx, const void *ws, uint32_t *dev_out, void *stream) {
    if (!ctx || !ws || !dev_out) return SIMULEE_EINVAL;
    const cudaError_t e = cudaMemcpyAsync(dev_out, (const uint8_t *)ws + offsetof(Ctl, hb_gbeg), sizeof(Ctl::hb_gbeg),
                                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
}

simulee_status simulee_set_stage_events(simulee_ctx *ctx, void *const *events, uint32_t n_events) {
    if (!ctx) return SIMULEE_EINVAL;
    if (!events || n_events == 0) {
        ctx->stage_on = false;
        return SIMULEE_OK;
    }
    if (n_events != 2 * SIMULEE_STAGES) return SIMULEE_EINVAL;
    for (uint32_t i = 0; i < n_events; i++) {
        if (!events[i]) return SIMULEE_EINVAL;
        ctx->stage_ev[i] = (cudaEvent_t)events[i];
    }
    ctx->stage_on = true;
    return SIMULEE_OK;
}

const char *simulee_status_str(simulee_status s) {
    switch (s) {
        case SIMULEE_OK: return "ok";
        case SIMULEE_EINVAL: return "invalid argument or dimensions out of range";
        case SIMULEE_EBADTRACE: return "invalid record or barrier count in the trace";
        case SIMULEE_ENOMEM: return "workspace too small (for the call, or for the records and races it met)";
        case SIMULEE_ETRUNC: return "an output held more records than its capacity";
        case SIMULEE_ETIMEOUT: return "a bounded device-side wait gave up";
        case SIMULEE_ECUDA: return "a CUDA call failed";
    }
    return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Check without a caller workspace, for callers that cannot allocate device
// memory. The scratch is this file-scope device array; host code must not use
// the array's name as an address (on the host it only names the symbol), so the
// device address is looked up with cudaGetSymbolAddress, once per device and
// primary context: the address is cached with the context it was found in, and
// looked up again when the device's current context is another one (the
// primary context was destroyed and created again, and the module with it).
// ---------------------------------------------------------------------------
static __device__ __align__(256) uint8_t g_noalloc_scratch[SIMULEE_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoallocEntry {
    void *context;   // the context the address was looked up in (nullptr: none yet)
    void *ptr;       // device address of the scratch array in that context
};
NoallocEntry g_noalloc[kNoallocMaxDevices];

// The calling thread's current driver context (cuCtxGetCurrent, reached through the runtime so that
// the library needs no link against the driver library), or nullptr when it cannot be told.
void *current_context() {
    using GetCurrent = CUresult (*)(CUcontext *);
    static std::once_flag once;
    static GetCurrent fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<GetCurrent>(f);
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return (void *)c;
}

// The scratch address on `device`; the caller has made `device` current. A lookup that is needed
// while `stream` is being captured is refused (EINVAL): the lookup may load the module, which a
// capture does not allow.
simulee_status noalloc_scratch(int device, cudaStream_t stream, void **ptr) {
    if (device < 0 || device >= kNoallocMaxDevices) return SIMULEE_EINVAL;
    void *context = current_context();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocEntry &e = g_noalloc[device];
    if (!e.ptr || !context || e.context != context) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return SIMULEE_ECUDA;
        if (cs != cudaStreamCaptureStatusNone) return SIMULEE_EINVAL;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SIMULEE_ECUDA;
        }
        e.context = context;
        e.ptr = p;
    }
    *ptr = e.ptr;
    return SIMULEE_OK;
}
}  // namespace

extern "C" simulee_status simulee_check_noalloc(simulee_ctx *ctx, const simulee_trace *trace,
                                                const simulee_outputs *out, simulee_report *report, void *stream) {
    if (!ctx || !trace) return SIMULEE_EINVAL;
    size_t need = 0;
    simulee_status s = simulee_workspace_size(ctx, trace, &need);
    if (s != SIMULEE_OK) return s;
    if (need > (size_t)SIMULEE_NOALLOC_SCRATCH_BYTES) return SIMULEE_ENOMEM;
    int prev_dev = -1;
    if (cudaGetDevice(&prev_dev) != cudaSuccess) return SIMULEE_ECUDA;
    // made current even when it already is: the device's primary context is then current too
    if (cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    void *scratch = nullptr;
    s = noalloc_scratch(ctx->device, (cudaStream_t)stream, &scratch);
    if (prev_dev != ctx->device) cudaSetDevice(prev_dev);
    if (s != SIMULEE_OK) return s;
    return simulee_check(ctx, trace, out, report, scratch, (size_t)SIMULEE_NOALLOC_SCRATCH_BYTES, stream);
}
