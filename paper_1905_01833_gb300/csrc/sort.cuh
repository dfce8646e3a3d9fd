// sort.cuh - hand-written onesweep LSD radix sort (one pass per 8-bit digit).
//
// Each pass is one persistent kernel. A CTA takes tiles of 4096 elements in
// the order it claims them (atomic tile counter), ranks its elements per
// digit (warp match + per-warp counters), publishes its per-digit counts,
// and finds the counts of all earlier tiles by decoupled look-back over a
// status array. A status word is (tag:8 | flag:2 | count:54), where the tag
// is the pass number of the current call, so words left over from an earlier
// pass are never mistaken for this pass's. Every wait on a predecessor is
// bounded by wall time (%globaltimer); a wait that gives up sets ctl->timeout,
// which makes every other waiter stop at once, and the call reports ETIMEOUT.
// Ranking within a tile is stable, tiles are ordered by claim order, so each
// pass is stable and the LSD sort is correct. With vin == vout == NULL the
// pass moves keys only.
#pragma once
#include "common.cuh"

namespace simk {

constexpr int OS_THREADS = 256;
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_ITEMS = 16;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;  // 4096
constexpr int OS_LOOKBACK = 4;                  // predecessor tiles read per look-back step

constexpr uint64_t ST_AGG = 1ull, ST_INC = 2ull;
__device__ __forceinline__ uint64_t st_make(uint32_t tag, uint64_t flag, uint64_t count) {
    return ((uint64_t)tag << 56) | (flag << 54) | count;
}
__device__ __forceinline__ uint32_t st_tag(uint64_t s) { return (uint32_t)(s >> 56); }
__device__ __forceinline__ uint64_t st_flag(uint64_t s) { return (s >> 54) & 3ull; }
__device__ __forceinline__ uint64_t st_count(uint64_t s) { return s & ((1ull << 54) - 1); }

// Shared memory of one pass: the tile's values and keys, then per digit the global bases, per digit the
// tile's exclusive offsets, per warp and digit the counts (16 bits: a tile holds at most 4096 elements; one
// column more for invalid lanes). With 16-bit counts a pass over 64-bit keys fits three CTAs per SM (72.7
// KB each; with 32-bit counts, 76.8 KB, only two).
template <class K, int ITEMS = OS_ITEMS, int BITS = RADIX_BITS>
constexpr size_t onesweep_smem() {
    constexpr size_t R = (size_t)1 << BITS, TILE = (size_t)OS_THREADS * ITEMS;
    return TILE * 8 + R * 8 + TILE * sizeof(K) + R * 4 + ((size_t)OS_WARPS * (R + 1) * 2 + 3) / 4 * 4;
}

// Block-wide exclusive scan of one value per thread (OS_THREADS threads).
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *warp_sums) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    uint32_t add = 0;
    for (int i = 0; i < w; i++) add += warp_sums[i];
    __syncthreads();
    return x - v + add;
}

// One LSD pass over digits of BITS bits (6 to 11) with tiles of OS_THREADS * ITEMS elements. Each
// thread owns DPT consecutive digits (one when BITS <= 8) for the per-digit steps: warp offsets,
// publication, look-back, global bases.
template <class K, int ITEMS = OS_ITEMS, int BITS = RADIX_BITS>
__global__ void __launch_bounds__(OS_THREADS, BITS > 8 ? 1 : 3)
k_onesweep(const K *__restrict__ kin, const uint64_t *__restrict__ vin, K *__restrict__ kout,
           uint64_t *__restrict__ vout, const uint32_t *n_ptr, uint64_t n_max, uint32_t shift,
           const uint32_t *__restrict__ dbase, unsigned long long *status, uint32_t tag, uint32_t *tile_ctr,
           Ctl *ctl, uint64_t wait_ns, uint32_t withhold, uint32_t tile_cap) {
    constexpr uint32_t R = 1u << BITS;
    constexpr int TILE = OS_THREADS * ITEMS;
    constexpr int DPT = (int)((R + OS_THREADS - 1) / OS_THREADS);
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *svals = reinterpret_cast<uint64_t *>(smem);                 // [TILE]
    uint64_t *gbase = svals + TILE;                                        // [R]
    K *skeys = reinterpret_cast<K *>(gbase + R);                           // [TILE]
    uint32_t *texcl = reinterpret_cast<uint32_t *>(skeys + TILE);          // [R]
    uint16_t *whist = reinterpret_cast<uint16_t *>(texcl + R);              // [OS_WARPS][R + 1]
    static_assert(OS_THREADS * ITEMS <= 65535 && ITEMS % 4 == 0, "16-bit digit counts, values loaded four at a time");
    __shared__ uint32_t wsum[OS_WARPS];
    __shared__ uint32_t s_tile;

    if (must_stop(ctl)) return;
    const uint64_t n = min((uint64_t)*n_ptr, n_max);
    if (n == 0) return;   // an empty stream (e.g. nothing left the hash path): no tile, no look-back
    // tile size: TILE elements, or, when there would be fewer tiles than mt (the grid's CTAs, at most
    // tile_cap when given), the smallest multiple of the CTA's threads that makes at most mt tiles
    // (the count is known on the device only; every CTA computes the same size). More, smaller tiles
    // mean less work per tile but longer look-back chains.
    uint32_t ipt = ITEMS;
    const uint64_t mt = tile_cap ? min((uint64_t)gridDim.x, (uint64_t)tile_cap) : (uint64_t)gridDim.x;
    if (n < mt * TILE) {
        const uint64_t per = mt * OS_THREADS;
        ipt = n > per ? (uint32_t)((n + per - 1) / per) : 1u;
    }
    const uint32_t tile_n = ipt * OS_THREADS;
    const uint64_t ntiles = (n + tile_n - 1) / tile_n;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = lanemask_lt();

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
        for (uint32_t i = tid; i < OS_WARPS * (R + 1); i += OS_THREADS) whist[i] = 0;
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles) return;
        const uint64_t base = tile * tile_n;
        const uint32_t nvalid = (uint32_t)min((uint64_t)tile_n, n - base);

        // element li of the tile: warp w holds li in [w * 32 * ipt, (w + 1) * 32 * ipt), item j of
        // lane l is li = w * 32 * ipt + j * 32 + l (items j >= ipt are unused)
        K k[ITEMS];
        uint32_t rd[ITEMS];   // rank within warp (low 16 bits) | digit << 16
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t li = w * (32 * ipt) + j * 32 + lane;
            k[j] = ((uint32_t)j < ipt && li < nvalid) ? kin[base + li] : K(0);
        }
        uint16_t *myhist = whist + w * (R + 1);
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            if ((uint32_t)j >= ipt) break;
            const uint32_t li = w * (32 * ipt) + j * 32 + lane;
            const bool valid = li < nvalid;
            const uint32_t d = valid ? (uint32_t)((k[j] >> shift) & (R - 1)) : R;
            // lanes holding the same digit: one ballot per digit bit (warp multi-split)
            const uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
            uint32_t peers = vmask;
#pragma unroll
            for (int bit = 0; bit < BITS; bit++) {
                const uint32_t on = (d >> bit) & 1u;
                const uint32_t m = __ballot_sync(0xFFFFFFFFu, on);
                peers &= on ? m : ~m;
            }
            if (!valid) peers = ~vmask;
            const uint32_t cnt = myhist[d];
            __syncwarp();
            if ((peers & lt) == 0) myhist[d] = (uint16_t)(cnt + __popc(peers));
            __syncwarp();
            rd[j] = (cnt + __popc(peers & lt)) | (d << 16);
        }
        __syncthreads();
        // per digit: exclusive offsets of the warps, tile count
        uint32_t run[DPT];
#pragma unroll
        for (int q = 0; q < DPT; q++) {
            const uint32_t d = (uint32_t)tid * DPT + q;
            uint32_t r = 0;
            if (d < R) {
#pragma unroll
                for (int ww = 0; ww < OS_WARPS; ww++) {
                    const uint32_t c = whist[ww * (R + 1) + d];
                    whist[ww * (R + 1) + d] = (uint16_t)r;
                    r += c;
                }
            }
            run[q] = r;
        }
        // publish this tile's counts, then look back over earlier tiles
        const bool withheld = withhold != 0 && tile == (uint64_t)(withhold - 1);
        volatile unsigned long long *vst = status;
#pragma unroll
        for (int q = 0; q < DPT; q++) {
            const uint32_t d = (uint32_t)tid * DPT + q;
            if (d < R && !withheld) vst[tile * R + d] = st_make(tag, tile == 0 ? ST_INC : ST_AGG, run[q]);
        }
#pragma unroll
        for (int q = 0; q < DPT; q++) {
            const uint32_t d = (uint32_t)tid * DPT + q;
            if (d >= R) continue;
            uint64_t excl = 0;
            if (tile > 0) {
                int64_t t = (int64_t)tile - 1;
                const uint64_t t0 = globaltimer_ns();
                uint32_t spins = 0;
                while (t >= 0) {
                    // four predecessors per step, their loads in flight together; consume them in order up
                    // to the first inclusive count, or up to a word not yet published (then read again)
                    uint64_t s4[OS_LOOKBACK];
#pragma unroll
                    for (int c = 0; c < OS_LOOKBACK; c++) s4[c] = t - c >= 0 ? vst[(uint64_t)(t - c) * R + d] : 0ull;
                    int used = 0;
                    bool inc = false, blocked = false;
#pragma unroll
                    for (int c = 0; c < OS_LOOKBACK; c++) {
                        if (inc || blocked || t - c < 0) continue;
                        const uint64_t sw = s4[c];
                        if (st_tag(sw) != tag || st_flag(sw) == 0) {
                            blocked = true;
                            continue;
                        }
                        excl += st_count(sw);
                        used = c + 1;
                        if (st_flag(sw) == ST_INC) inc = true;
                    }
                    if (inc) break;
                    t -= used;
                    if (blocked && (++spins & 63) == 0) {
                        if (*(volatile unsigned int *)&ctl->timeout) break;
                        if (globaltimer_ns() - t0 > wait_ns) {
                            atomicExch(&ctl->timeout, 1u);
                            break;
                        }
                    }
                }
                if (!withheld) vst[tile * R + d] = st_make(tag, ST_INC, excl + run[q]);
            }
            gbase[d] = (uint64_t)dbase[d] + excl;
        }
        // the tile's exclusive offsets per digit, in digit order
        uint32_t tsum = 0;
#pragma unroll
        for (int q = 0; q < DPT; q++) tsum += run[q];
        uint32_t acc = block_excl_scan_256(tsum, wsum);
#pragma unroll
        for (int q = 0; q < DPT; q++) {
            const uint32_t d = (uint32_t)tid * DPT + q;
            if (d < R) texcl[d] = acc;
            acc += run[q];
        }
        __syncthreads();
        // stable scatter into shared memory in digit order. The values are loaded four at a time, their
        // loads in flight together (one item at a time behind the item's bounds test, each load waited out
        // its whole latency: the pass was 18% slower)
        constexpr int VB = 4;
#pragma unroll
        for (int j0 = 0; j0 < ITEMS; j0 += VB) {
            uint64_t vv[VB];
#pragma unroll
            for (int jj = 0; jj < VB; jj++) {
                const int j = j0 + jj;
                const uint32_t li = w * (32 * ipt) + j * 32 + lane;
                vv[jj] = (vin && (uint32_t)j < ipt && li < nvalid) ? vin[base + li] : 0ull;
            }
#pragma unroll
            for (int jj = 0; jj < VB; jj++) {
                const int j = j0 + jj;
                const uint32_t li = w * (32 * ipt) + j * 32 + lane;
                if ((uint32_t)j < ipt && li < nvalid) {
                    const uint32_t d = rd[j] >> 16;
                    const uint32_t pos = texcl[d] + whist[w * (R + 1) + d] + (rd[j] & 0xFFFFu);
                    skeys[pos] = k[j];
                    if (vin) svals[pos] = vv[jj];
                }
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < nvalid; i += OS_THREADS) {
            const K kk = skeys[i];
            const uint32_t d = (uint32_t)((kk >> shift) & (R - 1));
            const uint64_t o = gbase[d] + (i - texcl[d]);
            if (o < n) {   // always true unless a wait gave up and the offsets are unreliable
                kout[o] = kk;
                if (vout) vout[o] = svals[i];
            }
        }
        __syncthreads();
    }
}

// Digit histograms of every pass of BITS-bit digits over a stream (count from the device), for the
// passes whose width the record reads do not histogram. Shared counts: npass * 2^BITS.
template <class K, int BITS>
__global__ void k_hist_keys(const K *__restrict__ keys, const uint32_t *n_ptr, uint64_t n_max, uint32_t npass,
                            uint32_t *hist, Ctl *ctl) {
    constexpr uint32_t R = 1u << BITS;
    extern __shared__ uint32_t hk_sh[];
    if (must_stop(ctl)) return;
    for (uint32_t i = threadIdx.x; i < npass * R; i += blockDim.x) hk_sh[i] = 0;
    __syncthreads();
    const uint64_t n = min((uint64_t)*n_ptr, n_max);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = (uint64_t)keys[i];
        for (uint32_t p = 0; p < npass; p++) atomicAdd(&hk_sh[p * R + ((uint32_t)(k >> (BITS * p)) & (R - 1))], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < npass * R; i += blockDim.x)
        if (hk_sh[i]) atomicAdd(&hist[i], hk_sh[i]);
}

// Exclusive scan of each pass's 2^BITS-digit histogram into its digit bases (one CTA per pass).
template <int BITS>
__global__ void k_digit_bases_w(const uint32_t *hist, uint32_t *dbase) {
    constexpr uint32_t R = 1u << BITS;
    constexpr int DPT = (int)((R + OS_THREADS - 1) / OS_THREADS);
    __shared__ uint32_t wsum[OS_WARPS];
    const uint32_t p = blockIdx.x;
    uint32_t v[DPT], tsum = 0;
#pragma unroll
    for (int q = 0; q < DPT; q++) {
        const uint32_t d = threadIdx.x * DPT + q;
        v[q] = d < R ? hist[p * R + d] : 0u;
        tsum += v[q];
    }
    uint32_t acc = block_excl_scan_256(tsum, wsum);
#pragma unroll
    for (int q = 0; q < DPT; q++) {
        const uint32_t d = threadIdx.x * DPT + q;
        if (d < R) dbase[p * R + d] = acc;
        acc += v[q];
    }
}

// Exclusive scan of each pass's histogram into its digit bases (one CTA per pass).
__global__ void k_digit_bases(const uint32_t *hist, uint32_t *dbase, Ctl *ctl) {
    __shared__ uint32_t wsum[OS_WARPS];
    const uint32_t p = blockIdx.x;
    const uint32_t v = hist[p * RADIX + threadIdx.x];
    const uint32_t e = block_excl_scan_256(v, wsum);
    dbase[p * RADIX + threadIdx.x] = e;
}

// Histograms of every digit pass of 64-bit keys (the race records), count from device.
__global__ void k_hist_u64(const uint64_t *keys, const uint32_t *n_ptr, uint64_t n_max, uint32_t npass,
                           uint32_t *hist, Ctl *ctl) {
    __shared__ uint32_t sh[8 * RADIX];
    if (must_stop(ctl)) return;
    for (int i = threadIdx.x; i < 8 * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t n = min((uint64_t)*n_ptr, n_max);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        for (uint32_t p = 0; p < npass; p++) atomicAdd(&sh[p * RADIX + ((k >> (8 * p)) & (RADIX - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)(npass * RADIX); i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

}  // namespace simk
