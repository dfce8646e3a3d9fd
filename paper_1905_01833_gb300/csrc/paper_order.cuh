// paper_order.cuh - the paper's visit-order counters (Algorithm 3, Sec. 3.2.2) for traces with
// flag PAPER_ORDER.
//
// Algorithm 3 keeps one counter per memory address, restarted for every block (global memory
// included); an access takes the counter's value, and a barrier bumps the counter only if the
// address was visited since its last bump. An access's visit order is therefore the number of
// earlier epochs in which its block touched its unit. Inside a block, grouping by visit order is
// grouping by epoch, so the intra-block streams are unchanged (only the adjacency test looks at
// the unit's next non-empty epoch, in k_reduce_groups). Across blocks, global accesses meet only
// at equal visit orders: the inter-block elements of such a trace are keyed (trace, visit order,
// unit) and built here from the global intra-block stream, once it is sorted by
// (block, unit, epoch): the visit order of an element is the number of distinct epochs before it
// within its (block, unit) run, a segmented count of group heads.
//
// One persistent kernel, tiles of 2048 elements claimed in order; the count carries across tiles
// by decoupled look-back over the status array (its own tag, distinct from every sort pass), with
// bounded waits as in the sort.
#pragma once
#include "check_kernels.cuh"
#include "sort.cuh"

namespace simk {

constexpr int PX_THREADS = 256;
constexpr int PX_ITEMS = 8;
constexpr int PX_TILE = PX_THREADS * PX_ITEMS;
constexpr uint32_t PX_TAG = 255;   // look-back tag of the visit-order scan
static_assert(MAX_PASSES < (int)PX_TAG, "sort passes use tags 1..MAX_PASSES");

// a segmented count: c = group heads since the last run head, f = a run head lies in the span
struct SegCount {
    uint32_t c, f;
};
// a followed by b
__device__ __forceinline__ SegCount seg_join(SegCount a, SegCount b) {
    return b.f ? b : SegCount{a.c + b.c, a.f};
}
__device__ __forceinline__ uint64_t seg_pack(SegCount s) { return (uint64_t)s.c | ((uint64_t)s.f << 40); }
__device__ __forceinline__ SegCount seg_unpack(uint64_t v) {
    return SegCount{(uint32_t)(v & 0xFFFFFFFFull), (uint32_t)((v >> 40) & 1u)};
}

template <class KG, class KX>
__global__ void __launch_bounds__(PX_THREADS)
k_paper_x(const KG *__restrict__ gk, const uint64_t *__restrict__ gv, const uint32_t *n_ptr, Layout L,
          const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, unsigned long long *status, Ctl *ctl,
          KX *xk, uint64_t *xv, uint64_t wait_ns) {
    __shared__ uint32_t s_tile;
    __shared__ SegCount s_warp[PX_THREADS / 32];
    __shared__ SegCount s_prefix;
    if (must_stop(ctl)) return;
    const uint64_t n = min((uint64_t)*n_ptr, L.cap_s);
    const uint64_t ntiles = (n + PX_TILE - 1) / PX_TILE;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t be = L.be;
    const uint64_t umask = (1ull << L.bug) - 1;
    volatile unsigned long long *vst = status;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctl->px_tile, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles) return;
        // thread tid holds the consecutive elements i0 .. i0 + PX_ITEMS - 1
        const uint64_t i0 = tile * PX_TILE + (uint64_t)tid * PX_ITEMS;
        uint64_t prev = (i0 > 0 && i0 - 1 < n) ? (uint64_t)gk[i0 - 1] : 0;
        uint32_t cj[PX_ITEMS];
        uint32_t fj = 0;   // bit j: a run head among items 0..j
        SegCount run{0, 0};
#pragma unroll
        for (int j = 0; j < PX_ITEMS; j++) {
            const uint64_t i = i0 + j;
            const bool in = i < n;
            const uint64_t k = in ? (uint64_t)gk[i] : 0;
            const bool head = in && (i == 0 || k != prev);                   // a new (block, unit, epoch) group
            const bool rhead = in && (i == 0 || (k >> be) != (prev >> be));  // a new (block, unit) run
            run = seg_join(run, SegCount{head ? 1u : 0u, rhead ? 1u : 0u});
            cj[j] = run.c;
            fj |= run.f << j;
            prev = k;
        }
        // exclusive scan of the threads' totals: inside the warp, then over the warps
        SegCount x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yc = __shfl_up_sync(0xFFFFFFFFu, x.c, o), yf = __shfl_up_sync(0xFFFFFFFFu, x.f, o);
            if (lane >= o) x = seg_join(SegCount{yc, yf}, x);
        }
        SegCount lex{__shfl_up_sync(0xFFFFFFFFu, x.c, 1), __shfl_up_sync(0xFFFFFFFFu, x.f, 1)};
        if (lane == 0) lex = SegCount{0, 0};
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        SegCount wex{0, 0}, tot{0, 0};
        for (int q = 0; q < PX_THREADS / 32; q++) {
            if (q == w) wex = tot;
            tot = seg_join(tot, s_warp[q]);
        }
        // the tile's prefix: decoupled look-back over the earlier tiles (thread 0)
        if (tid == 0) {
            vst[tile] = st_make(PX_TAG, tile == 0 ? ST_INC : ST_AGG, seg_pack(tot));
            SegCount acc{0, 0};
            if (tile > 0) {
                int64_t t = (int64_t)tile - 1;
                const uint64_t t0 = globaltimer_ns();
                uint32_t spins = 0;
                while (t >= 0) {
                    const uint64_t s = vst[t];
                    if (st_tag(s) != PX_TAG || st_flag(s) == 0) {
                        if ((++spins & 63) == 0) {
                            if (*(volatile unsigned int *)&ctl->timeout) break;
                            if (globaltimer_ns() - t0 > wait_ns) {
                                atomicExch(&ctl->timeout, 1u);
                                break;
                            }
                        }
                        continue;
                    }
                    acc = seg_join(seg_unpack(st_count(s)), acc);
                    if (st_flag(s) == ST_INC || acc.f) break;   // a run head: nothing earlier matters
                    --t;
                }
                vst[tile] = st_make(PX_TAG, ST_INC, seg_pack(seg_join(acc, tot)));
            }
            s_prefix = acc;
        }
        __syncthreads();
        const SegCount tpre = seg_join(seg_join(s_prefix, wex), lex);   // everything before this thread's items
        // the elements of paper-counter traces become inter-block elements keyed (trace, visit order, unit)
#pragma unroll
        for (int j = 0; j < PX_ITEMS; j++) {
            const uint64_t i = i0 + j;
            bool emit = false;
            uint64_t key = 0, val = 0;
            if (i < n) {
                const uint64_t k = (uint64_t)gk[i];
                const uint64_t sb = k >> (L.bug + be);
                const uint32_t t = tob[sb];
                const TraceDesc &d = td[t];
                if (d.flags & TF_PAPER_ORDER) {
                    const uint32_t count = ((fj >> j) & 1u) ? cj[j] : tpre.c + cj[j];
                    // the run's first group is visit order 0 (the mask keeps a count that a wait gave up on
                    // inside its field)
                    const uint32_t vord = (count - 1) & (uint32_t)((1ull << L.bxr) - 1);
                    const uint64_t v = gv[i];
                    const uint32_t gtid = (uint32_t)(v >> 32) & 0x3FFFFFFFu;
                    const uint32_t blk = gtid / d.bt, tt = gtid - blk * d.bt;
                    const uint32_t xo = d.nb <= (1u << 20) ? ((blk << 10) | tt) : gtid;
                    key = shl(t, L.bug + L.bxr) | ((uint64_t)vord << L.bug) | ((k >> be) & umask);
                    val = make_payload(payload_act(v), xo, (uint32_t)v);
                    emit = true;
                }
            }
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, emit);
            if (m) {
                uint32_t b0 = 0;
                if (lane == __ffs(m) - 1) b0 = atomicAdd(&ctl->n_x, (uint32_t)__popc(m));
                b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(m) - 1);
                if (emit) {
                    const uint64_t o = (uint64_t)b0 + __popc(m & lt);
                    if (o < L.x_cap) {
                        xk[o] = (KX)key;
                        xv[o] = val;
                    }
                }
            }
        }
        __syncthreads();   // s_warp and s_prefix are rewritten by the next tile
    }
}

}  // namespace simk
