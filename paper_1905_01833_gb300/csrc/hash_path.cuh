// hash_path.cuh - short-interval path: intra-block checks without sorting.
//
// Applies to traces whose records come in schedule order block by block and,
// inside a block, epoch by epoch (the order Algorithm 3's simulator emits),
// with at most HB_RUNMAX records per (block, epoch) run. One CTA takes a block
// and walks its epochs in order. The records of a run are grouped by memory
// unit in a shared-memory hash table (open addressing, Fibonacci hashing);
// per slot and category {read, write, atomic} two atomicMin passes give the
// earliest item and the earliest item of another thread (the top-2 summary of
// common.cuh), from which the slot's lowest conflicting pairs follow. The
// previous epoch's table keeps its keys and a packed adjacency summary per
// slot, so each unit of epoch e is tested against the same unit of epoch e-1
// (barrier e-1 needed or redundant) without a second pass over memory.
//
// The thread that creates a slot (wins the insert) finalises it, and resets it
// once it is no longer needed, so the work per epoch follows the number of
// distinct units rather than the table size. Each record is read once.
#pragma once
#include "check_kernels.cuh"

namespace simk {

constexpr int HB_THREADS = 1024;
constexpr int HB_RUNMAX = 2048;                     // records per (block, epoch) run
constexpr int HB_SLOTS = 4096;                      // load factor <= 1/2
constexpr int HB_PER_THREAD = HB_RUNMAX / HB_THREADS;
constexpr uint32_t HB_EMPTY = 0xFFFFFFFFu;
constexpr uint32_t HB_NO_OWNER = 0x7FFu;            // packed owner code: category absent

// shared memory: keys of two epochs, first/second items per category, adjacency summaries,
// and the staging buffer that receives the next run's records
constexpr size_t hash_blocks_smem() {
    return (size_t)HB_SLOTS * 4 * (2 + 3 + 3) + (size_t)HB_SLOTS * 8 + (size_t)HB_RUNMAX * 16;
}

__device__ __forceinline__ uint32_t hb_hash(uint32_t key) { return (key * 0x9E3779B1u) >> (32 - 12); }

// packed adjacency summary: x = ownR | ownW << 11 | multi << 22, y = ownA (owner = tid, 0x7FF = absent)
__device__ __forceinline__ uint2 hb_pack(const Top2 &s) {
    uint32_t own[3], multi = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        own[c] = s.a[c] == EMPTY ? HB_NO_OWNER : ((uint32_t)s.a[c] & 0x3FFu);
        if (s.b[c] != EMPTY) multi |= 1u << c;
    }
    return make_uint2(own[0] | (own[1] << 11) | (multi << 22), own[2]);
}

__device__ __forceinline__ bool hb_conflict(uint2 P, uint2 Q) {
    const uint32_t po[3] = {P.x & 0x7FFu, (P.x >> 11) & 0x7FFu, P.y & 0x7FFu};
    const uint32_t qo[3] = {Q.x & 0x7FFu, (Q.x >> 11) & 0x7FFu, Q.y & 0x7FFu};
    const uint32_t pm = (P.x >> 22) & 7u, qm = (Q.x >> 22) & 7u;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        if (po[i] == HB_NO_OWNER) continue;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (qo[j] == HB_NO_OWNER) continue;
            if ((i == 0 && j == 0) || (i == 2 && j == 2)) continue;   // read/read, atomic/atomic
            if (((pm >> i) & 1u) || ((qm >> j) & 1u) || po[i] != qo[j]) return true;
        }
    }
    return false;
}

// item of the table: run position << 10 | tid  ->  summary item: position << 32 | tid
__device__ __forceinline__ uint64_t hb_item64(uint32_t v) {
    return v == HB_EMPTY ? EMPTY : (((uint64_t)(v >> 10) << 32) | (v & 0x3FFu));
}

__global__ void __launch_bounds__(HB_THREADS, 1)
k_hash_blocks(const TraceDesc *__restrict__ td, const uint32_t *__restrict__ tob, const uint4 *__restrict__ stats,
              const uint32_t *__restrict__ runs, const uint32_t *__restrict__ binel, Layout L, TState *ts, Ctl *ctl,
              uint32_t *nonred, RaceStage rs, uint64_t wait_ns) {
    extern __shared__ __align__(128) uint32_t hb_smem[];
    uint4 *hrec = reinterpret_cast<uint4 *>(hb_smem);                      // [HB_RUNMAX] staged records
    uint32_t *hkey = hb_smem + HB_RUNMAX * 4;                              // [2][HB_SLOTS]
    uint32_t *hfirst = hkey + 2 * HB_SLOTS;                                // [3][HB_SLOTS]
    uint32_t *hsecond = hfirst + 3 * HB_SLOTS;                             // [3][HB_SLOTS]
    uint2 *hadj = reinterpret_cast<uint2 *>(hsecond + 3 * HB_SLOTS);       // [HB_SLOTS]
    __shared__ uint64_t bar;
    __shared__ uint32_t s_needed;   // barrier e-1 already found needed in this epoch
    const int tid = threadIdx.x;
    for (int i = tid; i < 8 * HB_SLOTS; i += HB_THREADS) hkey[i] = HB_EMPTY;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;   // completed copies into hrec, mod 2 (same value in every thread)
    const OwnThread own;
    for (uint64_t b = blockIdx.x; b < L.NB; b += gridDim.x) {
        const uint32_t t = tob[b];
        const TraceDesc &d = td[t];
        // uniform over the CTA: only suitable, valid hash-path traces
        if (!d.hash_ok || *(volatile uint32_t *)&ts[t].inel || binel[b] || trace_bad(ts[t])) continue;
        const uint64_t lb = b - d.block_off;
        const uint32_t maxc = min(stats[b].w, L.maxb);
        int cur = 0;
        bool prev_live = false;
        uint32_t mine_prev[HB_PER_THREAD], mine[HB_PER_THREAD];
#pragma unroll
        for (int j = 0; j < HB_PER_THREAD; j++) mine_prev[j] = HB_EMPTY;
        const uint64_t rbase = 2 * (uint64_t)b * (L.maxb + 1);
        // run bounds of epoch e of this block (empty when out of range)
        auto run_of = [&](uint32_t e, uint32_t &rs_, uint32_t &m_) {
            rs_ = 0;
            m_ = 0;
            if (e > maxc) return;
            const uint32_t a = runs[rbase + 2 * e], z = runs[rbase + 2 * e + 1];
            rs_ = a;
            m_ = (z > a) ? min(z - a, (uint32_t)HB_RUNMAX) : 0u;
        };
        // thread 0: start the copy of a run's records into hrec (hrec is free)
        auto prefetch = [&](uint32_t rs_, uint32_t m_) {
            if (m_ == 0) return;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar, m_ * 16u);
            bulk_g2s(hrec, d.events + rs_, m_ * 16u, &bar);
        };
        uint32_t rs0, m;
        run_of(0, rs0, m);
        if (tid == 0) prefetch(rs0, m);
        for (uint32_t e = 0; e <= maxc; e++) {
            uint32_t *key = hkey + cur * HB_SLOTS;
            const uint32_t *pkey = hkey + (cur ^ 1) * HB_SLOTS;
            uint32_t slot[HB_PER_THREAD], item[HB_PER_THREAD], cat[HB_PER_THREAD];
            if (m > 0) {
                const bool arrived = __syncthreads_and(mbar_wait(&bar, phase, wait_ns));
                if (!arrived) {
                    if (tid == 0) {
                        atomicExch(&ctl->timeout, 1u);
                        mbar_wait(&bar, phase, wait_ns);   // bounded: let the copy in flight land
                    }
                    return;
                }
                phase ^= 1u;
            }
            uint32_t rs1, m1;   // the next epoch's run
            run_of(e + 1, rs1, m1);
            // 1. insert this run's units; remember the slots this thread creates
#pragma unroll
            for (int j = 0; j < HB_PER_THREAD; j++) {
                mine[j] = HB_EMPTY;
                slot[j] = HB_EMPTY;
                const uint32_t r = tid + j * HB_THREADS;
                const uint4 ev = r < m ? hrec[r] : make_uint4(0, 0, 0, 0x30000000u);
                const uint32_t sp = (ev.w >> 30) & 1u;
                // fields were validated by the ingest; the check keeps shared memory safe regardless
                if (r < m && ((ev.w >> 28) & 3u) != 3u && ev.x < (sp ? d.gu : d.su)) {
                    const uint32_t k = (ev.x << 1) | sp;
                    item[j] = (r << 10) | (ev.w & 0x3FFu);
                    cat[j] = (ev.w >> 28) & 3u;
                    uint32_t s = hb_hash(k);
                    for (;;) {
                        const uint32_t cur_k = key[s];
                        if (cur_k == k) break;
                        if (cur_k == HB_EMPTY) {
                            const uint32_t old = atomicCAS(&key[s], HB_EMPTY, k);
                            if (old == HB_EMPTY) { mine[j] = s; break; }
                            if (old == k) break;
                        }
                        s = (s + 1) & (HB_SLOTS - 1);
                    }
                    slot[j] = s;
                }
            }
            if (tid == 0) s_needed = 0u;
            __syncthreads();
            if (tid == 0) prefetch(rs1, m1);   // every thread is done with hrec
            // 2. earliest item per slot and category, then the earliest of another thread
#pragma unroll
            for (int j = 0; j < HB_PER_THREAD; j++)
                if (slot[j] != HB_EMPTY) atomicMin(&hfirst[cat[j] * HB_SLOTS + slot[j]], item[j]);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < HB_PER_THREAD; j++)
                if (slot[j] != HB_EMPTY) {
                    const uint32_t f = hfirst[cat[j] * HB_SLOTS + slot[j]];
                    if ((f & 0x3FFu) != (item[j] & 0x3FFu)) atomicMin(&hsecond[cat[j] * HB_SLOTS + slot[j]], item[j]);
                }
            __syncthreads();
            // 3. creators finalise their slots: races, adjacency with the previous epoch
            bool needed = false;
            uint2 adj[HB_PER_THREAD];
#pragma unroll
            for (int j = 0; j < HB_PER_THREAD; j++) {
                const uint32_t s = mine[j];
                if (s == HB_EMPTY) continue;
                Top2 S;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    S.a[c] = hb_item64(hfirst[c * HB_SLOTS + s]);
                    S.b[c] = hb_item64(hsecond[c * HB_SLOTS + s]);
                }
                const uint32_t k = key[s];
                const uint32_t unit = k >> 1, space = k & 1u;
                const bool two_owners = S.b[0] != EMPTY || S.b[1] != EMPTY || S.b[2] != EMPTY ||
                                        (S.a[0] != EMPTY && S.a[1] != EMPTY && (uint32_t)S.a[0] != (uint32_t)S.a[1]) ||
                                        (S.a[0] != EMPTY && S.a[2] != EMPTY && (uint32_t)S.a[0] != (uint32_t)S.a[2]) ||
                                        (S.a[1] != EMPTY && S.a[2] != EMPTY && (uint32_t)S.a[1] != (uint32_t)S.a[2]);
                if (two_owners) {
#pragma unroll
                    for (int cls = 0; cls < 2; cls++) {
                        uint64_t p, q;
                        if (!lowest_pair(S, cls, own, p, q)) continue;
                        const uint32_t vp = d.events[rs0 + item_pos(p)].y, vq = d.events[rs0 + item_pos(q)].y;
                        const uint64_t pp = ((uint64_t)vp << 32) | (uint32_t)(lb * d.bt + item_gtid(p));
                        const uint64_t qq = ((uint64_t)vq << 32) | (uint32_t)(lb * d.bt + item_gtid(q));
                        emit_race(rs, ctl, t, race_key(L, t, space, 0u, (uint32_t)b, e, unit, cls), pp, qq);
                    }
                }
                adj[j] = hb_pack(S);
                if (prev_live && !needed && !*(volatile uint32_t *)&s_needed) {
                    uint32_t ps = hb_hash(k);
                    for (;;) {
                        const uint32_t pk = pkey[ps];
                        if (pk == HB_EMPTY) break;
                        if (pk == k) {
                            if (hb_conflict(hadj[ps], adj[j])) {
                                needed = true;
                                s_needed = 1u;
                            }
                            break;
                        }
                        ps = (ps + 1) & (HB_SLOTS - 1);
                    }
                }
            }
            if (__syncthreads_or(needed) && tid == 0) mark_needed(nonred, L, (uint32_t)b, e - 1);
            // 4. publish this epoch's summaries; release the previous epoch's keys and this epoch's items
#pragma unroll
            for (int j = 0; j < HB_PER_THREAD; j++) {
                const uint32_t s = mine[j];
                if (s != HB_EMPTY) {
                    hadj[s] = adj[j];
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        hfirst[c * HB_SLOTS + s] = HB_EMPTY;
                        hsecond[c * HB_SLOTS + s] = HB_EMPTY;
                    }
                }
                if (mine_prev[j] != HB_EMPTY) hkey[(cur ^ 1) * HB_SLOTS + mine_prev[j]] = HB_EMPTY;
                mine_prev[j] = mine[j];
            }
            __syncthreads();
            prev_live = m > 0;
            cur ^= 1;
            rs0 = rs1;
            m = m1;
        }
        // release the last epoch's keys before the next block
#pragma unroll
        for (int j = 0; j < HB_PER_THREAD; j++)
            if (mine_prev[j] != HB_EMPTY) hkey[(cur ^ 1) * HB_SLOTS + mine_prev[j]] = HB_EMPTY;
        __syncthreads();
    }
}

// A block with a (block, epoch) run longer than HB_RUNMAX records goes to the sort path.
__global__ void k_runs_check(const TraceDesc *td, const uint32_t *tob, const uint32_t *runs, Layout L,
                             uint32_t *binel) {
    const uint64_t tot = (uint64_t)L.NB * (L.maxb + 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = i / (L.maxb + 1);
        if (!td[tob[b]].hash_ok) continue;
        const uint32_t s = runs[2 * i], e = runs[2 * i + 1];
        if (e < s || e - s > (uint32_t)HB_RUNMAX) atomicOr(&binel[b], 1u);
    }
}

}  // namespace simk
