// fitness.cuh - the fitness of Eq. 1 (Sec. 3.3.1) for a batch of traces.
//
// For memory address i, f(i) is the number of distinct threads that access it
// and g(i) = 1 when it is accessed; F = sum g / sum f (1: no two threads share
// an address; smaller: more sharing, more chances of a conflict). An address
// is a global unit or a shared unit of one block; a thread is its global id;
// every epoch and action counts. The secondary fitness R = end - start uses
// the accessed unit range, reported per space.
//
// Both sums are distinct counts, found by sorting: every record becomes the
// key (trace | space | block for shared | unit | gtid), the keys are radix
// sorted (keys only), and the heads of equal keys count the distinct
// (address, thread) pairs while the heads of equal keys without the gtid
// field count the distinct addresses. Validation is the check's (barrier
// counts, then every record), so a bad trace reports the same first bad index.
#pragma once
#include "check_kernels.cuh"

namespace simk {

struct FitAcc {
    unsigned long long n_addr, n_pairs;
    unsigned int lo[2], hi[2];   // accessed unit range per space (lo > hi: none)
};

// key fields, low to high: gtid (bg) | unit (bu) | block for shared records (bbl) | space (1) | trace (btr)
struct FitKeys {
    uint32_t bg, bu, bbl, btr, bits, np;
};

constexpr int FK_THREADS = 256;
constexpr uint32_t FIT_OUT_BYTES = 48;   // sizeof(simulee_fitness)
constexpr int FK_ITEMS = IN_TILE / FK_THREADS;   // tiles never span traces

__global__ void k_fit_init(FitAcc *acc, uint32_t T) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        acc[t].n_addr = 0;
        acc[t].n_pairs = 0;
        acc[t].lo[0] = acc[t].lo[1] = 0xFFFFFFFFu;
        acc[t].hi[0] = acc[t].hi[1] = 0;
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

// keys, digit histograms and the per-space unit ranges; one tile (2048 records of one trace) at a time
template <class K>
__global__ void __launch_bounds__(FK_THREADS)
k_fit_keys(const TraceDesc *__restrict__ td, Layout L, FitKeys fk, K *keys, uint32_t *hist, FitAcc *acc) {
    __shared__ uint32_t sh[8 * RADIX];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < 8 * RADIX; i += FK_THREADS) sh[i] = 0;
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < L.ntiles_in; tile += gridDim.x) {
        const uint32_t t = trace_of_tile(td, L.T, tile);
        const TraceDesc &d = td[t];
        const uint64_t tbase = (tile - d.tile_off) * IN_TILE;
        uint32_t lo[2] = {0xFFFFFFFFu, 0xFFFFFFFFu}, hi[2] = {0, 0};
#pragma unroll 4
        for (int j = 0; j < FK_ITEMS; j++) {
            const uint64_t idx = tbase + j * FK_THREADS + tid;
            const bool in = idx < d.n;
            const uint4 e = in ? d.events[idx] : make_uint4(0, 0, 0, 0);
            const uint32_t sp = (e.w >> 30) & 1u, tt = e.w & 0xFFFFu;
            const uint64_t k = fit_key(fk, t, sp, e.z, e.x, e.z * d.bt + tt);
            if (in) {
                keys[d.rec_off + idx] = (K)k;
                lo[sp] = min(lo[sp], e.x);
                hi[sp] = max(hi[sp], e.x);
            }
            hist_add(sh, k, fk.np, in, __ballot_sync(0xFFFFFFFFu, in));
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
