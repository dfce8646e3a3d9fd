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
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/simulee.h"
#include "check_kernels.cuh"
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

simulee_status check_trace_args(const simulee_trace *t) {
    if (!t) return SIMULEE_EINVAL;
    if (t->n_events > 0 && !t->events) return SIMULEE_EINVAL;
    if (!t->barrier_counts) return SIMULEE_EINVAL;
    if (t->n_events >= (1ull << 31)) return SIMULEE_EINVAL;
    if (t->n_blocks == 0 || t->block_threads == 0 || t->block_threads > 1024) return SIMULEE_EINVAL;
    if ((uint64_t)t->n_blocks * t->block_threads > (1ull << 30)) return SIMULEE_EINVAL;
    if (t->max_barriers > 4095) return SIMULEE_EINVAL;
    if (t->flags & ~SIMULEE_FLAG_UNSORTED) return SIMULEE_EINVAL;
    if (((uintptr_t)t->events & 15u) != 0 || ((uintptr_t)t->barrier_counts & 3u) != 0) return SIMULEE_EINVAL;
    return SIMULEE_OK;
}

// Bit layouts, pass counts and workspace offsets for one trace.
simulee_status make_layout(const simulee_trace *t, Layout &L) {
    memset(&L, 0, sizeof L);
    L.n = t->n_events;
    L.nb = t->n_blocks;
    L.bt = t->block_threads;
    L.su = t->shared_units;
    L.gu = t->global_units;
    L.maxb = t->max_barriers;
    L.flags = t->flags;
    L.bb = bits_for(L.nb);
    L.bus = bits_for(L.su);
    L.bug = bits_for(L.gu);
    L.be = bits_for((uint64_t)L.maxb + 1);
    L.bu = std::max(L.bus, L.bug);
    L.bits_s = L.bb + L.bus + L.be;
    L.bits_g = L.bb + L.bug + L.be;
    L.bits_x = L.bug;
    L.bits_r = 3 + L.bb + L.be + L.bu;
    if (L.bits_s > 64 || L.bits_g > 64 || L.bits_r > 64) return SIMULEE_EINVAL;
    L.wide_s = L.bits_s > 32;
    L.wide_g = L.bits_g > 32;
    L.np_s = passes_for(L.bits_s);
    L.np_g = passes_for(L.bits_g);
    L.np_x = passes_for(L.bits_x);
    L.np_r = passes_for(L.bits_r);
    L.p0_s = 0;
    L.p0_g = L.p0_s + L.np_s;
    L.p0_x = L.p0_g + L.np_g;
    L.p0_r = L.p0_x + L.np_x;
    // the unsorted-trace rank sort uses passes p0_r + np_r .. + 3
    if (L.p0_r + L.np_r + 4 > MAX_PASSES) return SIMULEE_EINVAL;
    L.words = std::max<uint32_t>(1, (L.maxb + 31) / 32);
    L.race_cap = 2 * L.n + 2;
    const uint64_t n = std::max<uint64_t>(L.n, 1);
    const uint64_t sort_max = std::max<uint64_t>(n, L.race_cap);
    L.status_tiles = (sort_max + OS_TILE - 1) / OS_TILE;

    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
    L.off_ctl = take(sizeof(Ctl));
    L.off_stats = take((size_t)L.nb * 16);
    L.off_nonred = take((size_t)L.nb * L.words * 4);
    L.off_gridnr = take((size_t)L.words * 4);
    L.off_gridhas = take((size_t)L.words * 4);
    L.off_cnt_div = take((size_t)L.nb * 4);
    L.off_cnt_red = take((size_t)L.nb * 4);
    L.off_ofs_div = take((size_t)L.nb * 4);
    L.off_ofs_red = take((size_t)L.nb * 4);
    L.off_hist = take((size_t)MAX_PASSES * RADIX * 4);
    L.off_dbase = take((size_t)MAX_PASSES * RADIX * 4);
    L.off_status = take((size_t)L.status_tiles * RADIX * 8);
    const size_t ks = L.wide_s ? 8 : 4, kg = L.wide_g ? 8 : 4;
    for (int i = 0; i < 2; i++) {
        L.off_sk[i] = take(n * ks);
        L.off_sv[i] = take(n * 8);
        L.off_gk[i] = take(n * kg);
        L.off_gv[i] = take(n * 8);
        L.off_xk[i] = take(n * 4);
        L.off_xv[i] = take(n * 8);
        L.off_rk[i] = take(L.race_cap * 8);
        L.off_rv[i] = take(L.race_cap * 8);
    }
    L.off_rp = take(L.race_cap * 16);
    L.total = o;
    return SIMULEE_OK;
}

// extra workspace for unsorted traces: rank[n] and pos_to_vo[n]
size_t unsorted_extra(const Layout &L) {
    return (L.flags & SIMULEE_FLAG_UNSORTED) ? 2 * align_up(std::max<uint64_t>(L.n, 1) * 4) : 0;
}

template <class K>
void set_sort_attr() {
    cudaFuncSetAttribute(k_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem<K>());
}

template <class K, bool INTER>
void set_reduce_attr() {
    cudaFuncSetAttribute(k_reduce_groups<K, INTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)reduce_groups_smem<K, INTER>());
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

    int sort_grid(uint64_t n_max) const {
        const uint64_t tiles = (n_max + OS_TILE - 1) / OS_TILE;
        return (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)ctx->sms * 2));
    }

    // LSD sort of (key, value) pairs in buffers 0/1; returns the buffer holding the result.
    template <class K>
    int sort(size_t koff[2], size_t voff[2], const uint32_t *n_ptr, uint64_t n_max, uint32_t np, uint32_t p0) {
        const int grid = sort_grid(n_max);
        for (uint32_t p = 0; p < np; p++) {
            const int src = p & 1, dst = src ^ 1;
            const uint32_t wh = first_pass_done ? 0u : withhold;
            first_pass_done = true;
            k_onesweep<K><<<grid, OS_THREADS, onesweep_smem<K>(), st>>>(
                at<K>(koff[src]), at<uint64_t>(voff[src]), at<K>(koff[dst]), at<uint64_t>(voff[dst]), n_ptr, n_max,
                RADIX_BITS * p, at<uint32_t>(L.off_dbase) + (size_t)(p0 + p) * RADIX,
                at<unsigned long long>(L.off_status), p0 + p + 1, &ctl->tiles[p0 + p], ctl, wait_ns, wh);
            launches++;
        }
        return (int)(np & 1);
    }
};

__global__ void k_rank_init(const uint4 *ev, uint64_t n, uint32_t *keys, uint64_t *vals, uint32_t *hist) {
    __shared__ uint32_t sh[4 * RADIX];
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t vo = ev[i].y;
        keys[i] = vo;
        vals[i] = i;
        for (int p = 0; p < 4; p++) atomicAdd(&sh[p * RADIX + ((vo >> (8 * p)) & (RADIX - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void k_rank_scatter(const uint64_t *sorted_idx, uint64_t n, uint32_t *rank, Ctl *ctl) {
    if (must_stop(ctl)) return;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (sorted_idx[i] < n) rank[sorted_idx[i]] = (uint32_t)i;
}

__global__ void k_set_count(unsigned int *dst, unsigned int v) { *dst = v; }

simulee_status launch_check(simulee_ctx *ctx, const simulee_trace *t, const simulee_outputs *out, Want want,
                            simulee_report *report, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !out || !report || !ws) return SIMULEE_EINVAL;
    simulee_status s = check_trace_args(t);
    if (s != SIMULEE_OK) return s;
    if ((out->races_cap && !out->races) || (out->divergence_cap && !out->divergence) ||
        (out->redundant_cap && !out->redundant) || (out->grid_redundant_cap && !out->grid_redundant))
        return SIMULEE_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SIMULEE_EINVAL;
    Run R;
    R.ctx = ctx;
    s = make_layout(t, R.L);
    if (s != SIMULEE_OK) return s;
    const size_t extra = unsorted_extra(R.L);
    if (ws_bytes < R.L.total + extra) return SIMULEE_ENOMEM;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    if (!ctx->attrs_set) {
        set_sort_attr<uint32_t>();
        set_sort_attr<uint64_t>();
        set_reduce_attr<uint32_t, false>();
        set_reduce_attr<uint64_t, false>();
        set_reduce_attr<uint32_t, true>();
        ctx->attrs_set = true;
    }
    R.st = (cudaStream_t)stream;
    R.ws = (uint8_t *)ws;
    R.ctl = R.at<Ctl>(R.L.off_ctl);
    R.wait_ns = (uint64_t)(ctx->opt.wait_limit_us ? ctx->opt.wait_limit_us : 1000000u) * 1000ull;
    R.withhold = ctx->opt.test_withhold;
    const Layout &L = R.L;
    const int sms = ctx->sms;
    cudaStream_t st = R.st;

    // 1. zero control state
    cudaMemsetAsync(R.ws, 0, L.off_cnt_div, st);   // ctl, stats, bitmaps
    cudaMemsetAsync(R.ws + L.off_hist, 0, (size_t)MAX_PASSES * RADIX * 4, st);
    cudaMemsetAsync(R.ws + L.off_status, 0, (size_t)L.status_tiles * RADIX * 8, st);

    // 2. barrier counts
    R.mark(SIMULEE_STAGE_INGEST, 0);
    {
        const int grid = (int)std::min<uint64_t>((L.nb + 7) / 8, (uint64_t)sms * 16);
        k_block_stats<<<std::max(grid, 1), 256, 0, st>>>(t->barrier_counts, L, R.at<uint4>(L.off_stats), R.ctl);
        R.launches++;
    }

    const bool route = want.races || want.red;
    const bool sorting = L.n > 0 && route;
    uint32_t *rank = nullptr, *pos_to_vo = nullptr;
    uint32_t *hist = R.at<uint32_t>(L.off_hist);
    if (L.n > 0) {
        // 3. unsorted traces: schedule rank of each record = position in (visit order, index) order
        if (L.flags & SIMULEE_FLAG_UNSORTED) {
            rank = R.at<uint32_t>(L.total);
            pos_to_vo = R.at<uint32_t>(L.total + align_up(L.n * 4));
            const uint32_t p0q = L.p0_r + L.np_r;
            size_t qk[2] = {L.off_rk[0], L.off_rk[1]}, qv[2] = {L.off_rv[0], L.off_rv[1]};
            const int g = (int)std::min<uint64_t>((L.n + 255) / 256, (uint64_t)sms * 8);
            k_rank_init<<<g, 256, 0, st>>>((const uint4 *)t->events, L.n, R.at<uint32_t>(qk[0]),
                                            R.at<uint64_t>(qv[0]), hist + (size_t)p0q * RADIX);
            k_digit_bases<<<4, RADIX, 0, st>>>(hist + (size_t)p0q * RADIX,
                                               R.at<uint32_t>(L.off_dbase) + (size_t)p0q * RADIX, R.ctl);
            k_set_count<<<1, 1, 0, st>>>(&R.ctl->n_q, (unsigned int)L.n);
            R.launches += 3;
            const int b = R.sort<uint32_t>(qk, qv, &R.ctl->n_q, L.n, 4, p0q);
            k_rank_scatter<<<g, 256, 0, st>>>(R.at<uint64_t>(qv[b]), L.n, rank, R.ctl);
            R.launches++;
            cudaMemcpyAsync(pos_to_vo, R.at<uint32_t>(qk[b]), L.n * 4, cudaMemcpyDeviceToDevice, st);
        }

        // 4. ingest
        const uint64_t ntiles = (L.n + IN_TILE - 1) / IN_TILE;
        const int gi = (int)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)sms * 4));
#define SIM_INGEST(KS, KG, RT)                                                                                     \
    k_ingest<KS, KG, RT><<<gi, IN_THREADS, 0, st>>>((const uint4 *)t->events, t->barrier_counts, rank, L, R.ctl,  \
                                                    R.at<KS>(L.off_sk[0]), R.at<uint64_t>(L.off_sv[0]),             \
                                                    R.at<KG>(L.off_gk[0]), R.at<uint64_t>(L.off_gv[0]),             \
                                                    R.at<uint32_t>(L.off_xk[0]), R.at<uint64_t>(L.off_xv[0]), hist)
        if (!route) {
            SIM_INGEST(uint32_t, uint32_t, false);
        } else if (L.wide_s && L.wide_g) {
            SIM_INGEST(uint64_t, uint64_t, true);
        } else if (L.wide_s) {
            SIM_INGEST(uint64_t, uint32_t, true);
        } else if (L.wide_g) {
            SIM_INGEST(uint32_t, uint64_t, true);
        } else {
            SIM_INGEST(uint32_t, uint32_t, true);
        }
#undef SIM_INGEST
        R.launches++;
    }
    R.mark(SIMULEE_STAGE_INGEST, 1);

    // 5. sort the three streams
    R.mark(SIMULEE_STAGE_SORT, 0);
    int bs = 0, bg = 0, bx = 0;
    if (sorting) {
        if (L.p0_r > 0) {
            k_digit_bases<<<L.p0_r, RADIX, 0, st>>>(hist, R.at<uint32_t>(L.off_dbase), R.ctl);
            R.launches++;
        }
        size_t sk[2] = {L.off_sk[0], L.off_sk[1]}, sv[2] = {L.off_sv[0], L.off_sv[1]};
        size_t gk[2] = {L.off_gk[0], L.off_gk[1]}, gv[2] = {L.off_gv[0], L.off_gv[1]};
        size_t xk[2] = {L.off_xk[0], L.off_xk[1]}, xv[2] = {L.off_xv[0], L.off_xv[1]};
        bs = L.wide_s ? R.sort<uint64_t>(sk, sv, &R.ctl->n_s, L.n, L.np_s, L.p0_s)
                      : R.sort<uint32_t>(sk, sv, &R.ctl->n_s, L.n, L.np_s, L.p0_s);
        bg = L.wide_g ? R.sort<uint64_t>(gk, gv, &R.ctl->n_g, L.n, L.np_g, L.p0_g)
                      : R.sort<uint32_t>(gk, gv, &R.ctl->n_g, L.n, L.np_g, L.p0_g);
        bx = R.sort<uint32_t>(xk, xv, &R.ctl->n_g, L.n, L.np_x, L.p0_x);
    }
    R.mark(SIMULEE_STAGE_SORT, 1);

    // 6. segmented reductions
    R.mark(SIMULEE_STAGE_REDUCE, 0);
    RaceStage rs;
    rs.keys = R.at<uint64_t>(L.off_rk[0]);
    rs.idx = R.at<uint64_t>(L.off_rv[0]);
    rs.pay = R.at<uint4>(L.off_rp);
    rs.cap = L.race_cap;
    rs.pos_to_vo = pos_to_vo;
    rs.n_pos = L.n;
    if (sorting) {
        uint32_t *nonred = R.at<uint32_t>(L.off_nonred);
        const int gr = (int)std::max<uint64_t>(1, std::min<uint64_t>((L.n + RG_TILE - 1) / RG_TILE, (uint64_t)sms * 3));
        if (L.wide_s)
            k_reduce_groups<uint64_t, false><<<gr, RG_THREADS, reduce_groups_smem<uint64_t, false>(), st>>>(
                R.at<uint64_t>(L.off_sk[bs]), R.at<uint64_t>(L.off_sv[bs]), &R.ctl->n_s, L, 0u, L.bus, R.ctl, nonred, rs);
        else
            k_reduce_groups<uint32_t, false><<<gr, RG_THREADS, reduce_groups_smem<uint32_t, false>(), st>>>(
                R.at<uint32_t>(L.off_sk[bs]), R.at<uint64_t>(L.off_sv[bs]), &R.ctl->n_s, L, 0u, L.bus, R.ctl, nonred, rs);
        if (L.wide_g)
            k_reduce_groups<uint64_t, false><<<gr, RG_THREADS, reduce_groups_smem<uint64_t, false>(), st>>>(
                R.at<uint64_t>(L.off_gk[bg]), R.at<uint64_t>(L.off_gv[bg]), &R.ctl->n_g, L, 1u, L.bug, R.ctl, nonred, rs);
        else
            k_reduce_groups<uint32_t, false><<<gr, RG_THREADS, reduce_groups_smem<uint32_t, false>(), st>>>(
                R.at<uint32_t>(L.off_gk[bg]), R.at<uint64_t>(L.off_gv[bg]), &R.ctl->n_g, L, 1u, L.bug, R.ctl, nonred, rs);
        k_reduce_groups<uint32_t, true><<<gr, RG_THREADS, reduce_groups_smem<uint32_t, true>(), st>>>(R.at<uint32_t>(L.off_xk[bx]), R.at<uint64_t>(L.off_xv[bx]),
                                                                  &R.ctl->n_g, L, 1u, L.bug, R.ctl, nonred, rs);
        R.launches += 3;
    }
    R.mark(SIMULEE_STAGE_REDUCE, 1);

    // 7. races in canonical order
    R.mark(SIMULEE_STAGE_RACES, 0);
    if (sorting && want.races) {
        const int gh = (int)std::max<uint64_t>(1, std::min<uint64_t>((L.race_cap + 255) / 256, (uint64_t)sms * 4));
        k_hist_u64<<<gh, 256, 0, st>>>(rs.keys, &R.ctl->n_races, L.race_cap, L.np_r, hist + (size_t)L.p0_r * RADIX,
                                       R.ctl);
        k_digit_bases<<<L.np_r, RADIX, 0, st>>>(hist + (size_t)L.p0_r * RADIX,
                                                R.at<uint32_t>(L.off_dbase) + (size_t)L.p0_r * RADIX, R.ctl);
        R.launches += 2;
        size_t rk[2] = {L.off_rk[0], L.off_rk[1]}, rv[2] = {L.off_rv[0], L.off_rv[1]};
        const int br = R.sort<uint64_t>(rk, rv, &R.ctl->n_races, L.race_cap, L.np_r, L.p0_r);
        if (out->races_cap) {
            const int gw = (int)std::max<uint64_t>(
                1, std::min<uint64_t>((std::min<uint64_t>(out->races_cap, L.race_cap) + 255) / 256, (uint64_t)sms * 8));
            k_write_races<<<gw, 256, 0, st>>>(R.at<uint64_t>(rk[br]), R.at<uint64_t>(rv[br]), rs.pay, L, R.ctl,
                                              (uint8_t *)out->races, out->races_cap);
            R.launches++;
        }
    }
    R.mark(SIMULEE_STAGE_RACES, 1);

    // 8. per-block outputs
    R.mark(SIMULEE_STAGE_BLOCKS, 0);
    if (want.div || want.red) {
        const int gb = (int)std::max<uint64_t>(1, std::min<uint64_t>((L.nb + 255) / 256, (uint64_t)sms * 8));
        k_block_counts<<<gb, 256, 0, st>>>(R.at<uint4>(L.off_stats), R.at<uint32_t>(L.off_nonred), L, R.ctl,
                                           R.at<uint32_t>(L.off_cnt_div), R.at<uint32_t>(L.off_cnt_red));
        k_scan2<<<1, 1024, 0, st>>>(R.at<uint32_t>(L.off_cnt_div), R.at<uint32_t>(L.off_cnt_red), L.nb,
                                    R.at<uint32_t>(L.off_ofs_div), R.at<uint32_t>(L.off_ofs_red), &R.ctl->n_div,
                                    &R.ctl->n_red, R.ctl);
        k_block_write<<<gb, 256, 0, st>>>(R.at<uint4>(L.off_stats), R.at<uint32_t>(L.off_nonred), L, R.ctl,
                                          R.at<uint32_t>(L.off_ofs_div), R.at<uint32_t>(L.off_ofs_red),
                                          want.div ? (uint4 *)out->divergence : nullptr,
                                          want.div ? out->divergence_cap : 0,
                                          want.red ? (uint2 *)out->redundant : nullptr, want.red ? out->redundant_cap : 0);
        R.launches += 3;
        if (want.red) {
            const int gg = (int)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)L.nb * L.words + 255) / 256, (uint64_t)sms * 8));
            k_grid_or<<<gg, 256, 0, st>>>(R.at<uint4>(L.off_stats), R.at<uint32_t>(L.off_nonred), L, R.ctl,
                                          R.at<uint32_t>(L.off_gridnr), R.at<uint32_t>(L.off_gridhas));
            k_grid_list<<<1, 1024, 0, st>>>(R.at<uint32_t>(L.off_gridnr), R.at<uint32_t>(L.off_gridhas), L, R.ctl,
                                            out->grid_redundant, out->grid_redundant_cap);
            R.launches += 2;
        }
    }

    // 9. report
    ReportArgs ra;
    ra.cap_races = out->races_cap;
    ra.cap_div = out->divergence_cap;
    ra.cap_red = out->redundant_cap;
    ra.cap_grid = out->grid_redundant_cap;
    ra.want_races = want.races;
    ra.want_div = want.div;
    ra.want_red = want.red;
    k_report<<<1, 32, 0, st>>>(R.ctl, ra, (uint8_t *)report);
    R.launches++;
    R.mark(SIMULEE_STAGE_BLOCKS, 1);
    ctx->last_launches = R.launches;
    const cudaError_t e = cudaGetLastError();
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? SIMULEE_OK : SIMULEE_ECUDA;
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
    simulee_ctx *c = (simulee_ctx *)calloc(1, sizeof(simulee_ctx));
    if (!c) return SIMULEE_ENOMEM;
    c->device = device;
    c->sms = prop.multiProcessorCount;
    if (opt) c->opt = *opt;
    *ctx = c;
    return SIMULEE_OK;
}

simulee_status simulee_destroy(simulee_ctx *ctx) {
    if (!ctx) return SIMULEE_EINVAL;
    free(ctx);
    return SIMULEE_OK;
}

simulee_status simulee_workspace_size(simulee_ctx *ctx, const simulee_trace *trace, size_t *bytes) {
    if (!ctx || !trace || !bytes) return SIMULEE_EINVAL;
    if (trace->n_blocks == 0 || trace->block_threads == 0 || trace->block_threads > 1024 ||
        trace->max_barriers > 4095 || trace->n_events >= (1ull << 31))
        return SIMULEE_EINVAL;
    Layout L;
    const simulee_status s = make_layout(trace, L);
    if (s != SIMULEE_OK) return s;
    *bytes = L.total + unsorted_extra(L);
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
    (void)ctx; (void)traces; (void)n_traces; (void)bytes;
    return SIMULEE_EINVAL;
}

simulee_status simulee_check_batch(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                   const simulee_outputs *outs, simulee_report *reports, void *ws, size_t ws_bytes,
                                   void *stream) {
    (void)ctx; (void)traces; (void)n_traces; (void)outs; (void)reports; (void)ws; (void)ws_bytes; (void)stream;
    return SIMULEE_EINVAL;
}

uint32_t simulee_last_launches(const simulee_ctx *ctx) { return ctx ? ctx->last_launches : 0u; }

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
        case SIMULEE_ENOMEM: return "workspace too small";
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
// device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
static __device__ __align__(256) uint8_t g_noalloc_scratch[SIMULEE_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices];   // device address of the scratch per device, once looked up

// Looks up the scratch address on `device`; the caller has made `device` current.
simulee_status noalloc_scratch(int device, void **ptr) {
    if (device < 0 || device >= kNoallocMaxDevices) return SIMULEE_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SIMULEE_ECUDA;
        g_noalloc_ptr[device] = p;
    }
    *ptr = g_noalloc_ptr[device];
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
    if (prev_dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return SIMULEE_ECUDA;
    void *scratch = nullptr;
    s = noalloc_scratch(ctx->device, &scratch);
    if (prev_dev != ctx->device) cudaSetDevice(prev_dev);
    if (s != SIMULEE_OK) return s;
    return simulee_check(ctx, trace, out, report, scratch, (size_t)SIMULEE_NOALLOC_SCRATCH_BYTES, stream);
}
