// models.cuh - device trace generator of parametric model kernels, the inputs of the
// evolutionary search of Algorithm 1 (Sec. 3.3): a population of launch
// configurations (grid and block dimensions, integer arguments) becomes one
// batch of traces in one launch, ready for the batched fitness and the check.
//
// Each record is computed from its index alone (schedule order: block, epoch,
// slot, thread; visit order = index within the launch):
//   copy2d: 2-D blocks; thread (x, y) of block (bx, by) has X = bx * block_x + x,
//     Y = by * block_y + y; slot 0 reads global src[(Y * arg1 + X) mod 2^19],
//     slot 1 writes global dst[2^19 + (Y * arg0 + X) mod 2^19]; no barrier.
//   stencil: 1-D blocks; epoch 0: thread t writes shared sh[(t * arg1) mod 4096];
//     one barrier; epoch 1: slot 0 reads sh[(t * arg1 + arg0) mod 4096], slot 1
//     writes global out[(block * block_x + t) mod 2^20].
// Negative arguments count as 0.
#pragma once
#include "common.cuh"

namespace simk {

constexpr uint32_t MD_HALF = 1u << 19;
constexpr uint32_t MD_SHARED = 4096;
constexpr uint32_t MD_GLOBAL = 1u << 20;

__device__ __forceinline__ uint32_t md_pack_w3(uint32_t tid, uint32_t epoch, uint32_t act, uint32_t space) {
    return (tid & 0xFFFFu) | ((epoch & 0xFFFu) << 16) | (act << 28) | (space << 30);
}

__global__ void k_model_traces(const simulee_model *__restrict__ m, uint32_t n_models, uint64_t n_events,
                               uint4 *events, uint64_t n_counts, uint32_t *counts) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_events; r += stride) {
        const uint32_t c = find_trace(n_models, r, [&](uint32_t i) { return m[i].events_off; });
        const simulee_model &p = m[c];
        const uint64_t bt = (uint64_t)p.block_x * p.block_y;
        const uint64_t per_block = (p.model == SIMULEE_MODEL_COPY2D ? 2 : 3) * bt;
        const uint64_t lr = r - p.events_off;
        const uint64_t b = lr / per_block, rem = lr % per_block;
        const uint64_t slot = rem / bt, t = rem % bt;
        const uint64_t a0 = (uint64_t)max(p.arg0, 0), a1 = (uint64_t)max(p.arg1, 0);
        uint32_t unit, w3;
        if (p.model == SIMULEE_MODEL_COPY2D) {
            const uint64_t X = (b % p.grid_x) * p.block_x + t % p.block_x;
            const uint64_t Y = (b / p.grid_x) * p.block_y + t / p.block_x;
            if (slot == 0) {
                unit = (uint32_t)((Y * a1 + X) % MD_HALF);
                w3 = md_pack_w3((uint32_t)t, 0, ACT_R, 1);
            } else {
                unit = MD_HALF + (uint32_t)((Y * a0 + X) % MD_HALF);
                w3 = md_pack_w3((uint32_t)t, 0, ACT_W, 1);
            }
        } else {
            if (slot == 0) {
                unit = (uint32_t)((t * a1) % MD_SHARED);
                w3 = md_pack_w3((uint32_t)t, 0, ACT_W, 0);
            } else if (slot == 1) {
                unit = (uint32_t)((t * a1 + a0) % MD_SHARED);
                w3 = md_pack_w3((uint32_t)t, 1, ACT_R, 0);
            } else {
                unit = (uint32_t)((b * p.block_x + t) % MD_GLOBAL);
                w3 = md_pack_w3((uint32_t)t, 1, ACT_W, 1);
            }
        }
        events[r] = make_uint4(unit, (uint32_t)lr, (uint32_t)b, w3);
    }
    // barrier counts: per launch, every thread passes 0 (copy2d) or 1 (stencil) barriers
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_counts; i += stride) {
        const uint32_t c = find_trace(n_models, i, [&](uint32_t k) { return m[k].counts_off; });
        counts[i] = m[c].model == SIMULEE_MODEL_COPY2D ? 0u : 1u;
    }
}

}  // namespace simk
