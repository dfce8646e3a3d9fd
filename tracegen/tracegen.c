/*
 * tracegen.c - seeded synthetic memory-access traces.
 *
 * This module only SYNTHESISES inputs: it writes 16-byte access records and
 * per-thread barrier counts in the shapes of the workloads the detector is
 * measured on. It holds no part of the detection arithmetic, and both the CPU
 * oracle and the CUDA path consume what it writes.
 *
 * Record layout (four little-endian 32-bit words):
 *   w0 unit, w1 visit_order, w2 block,
 *   w3 = tid[0:16] | epoch[16:28] | action[28:30] | space[30] | reserved[31]
 *   action: 0 read, 1 write, 2 atomic;  space: 0 shared, 1 global.
 *
 * Randomness is counter based: every draw is a hash of (seed, purpose, and the
 * coordinates of the draw), so a record's content does not depend on the order
 * in which records are produced. The hash is the SplitMix64 output function
 * (Steele, Lea and Flood, OOPSLA 2014) applied as a mixer.
 *
 * Every generator returns the number of records. With ev == NULL it only
 * counts, so callers size buffers with a first call.
 */
#include <stdint.h>
#include <stddef.h>

#define ACT_R 0u
#define ACT_W 1u
#define ACT_A 2u
#define SP_SH 0u
#define SP_GL 1u

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* hash of a seed, a purpose tag and up to four coordinates */
static inline uint64_t hsh(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    uint64_t x = mix64(seed ^ (tag * 0xD1B54A32D192ED03ull));
    x = mix64(x ^ a);
    x = mix64(x ^ (b + 0x632BE59BD9B4E019ull));
    x = mix64(x ^ (c + 0x8CB92BA72F3D8DD7ull));
    x = mix64(x ^ (d + 0x52DCE729DA3ED4A1ull));
    return x;
}

/* uniform double in [0,1) from the top 53 bits */
static inline double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    uint32_t *ev;      /* NULL: count only */
    uint64_t n;        /* records emitted so far */
} sink;

static inline void emit(sink *s, uint32_t unit, uint32_t block, uint32_t tid, uint32_t epoch,
                        uint32_t act, uint32_t space) {
    if (s->ev) {
        uint32_t *r = s->ev + 4 * s->n;
        r[0] = unit;
        r[1] = (uint32_t)s->n;   /* visit order = serial position in the schedule */
        r[2] = block;
        r[3] = (tid & 0xFFFFu) | ((epoch & 0xFFFu) << 16) | ((act & 3u) << 28) | ((space & 1u) << 30);
    }
    s->n++;
}

/* ------------------------------------------------------------------------ */
/* Single block, strided shared-memory accesses.                            */
/*   n_threads threads, n_epochs epochs (barrier count n_epochs-1 each),    */
/*   per epoch a stride s in {1,2,32}; thread t issues k = 0..per_thread-1  */
/*   accesses at unit (t*s + k) mod shared_units, writes with probability   */
/*   write_p, and with probability redirect_p takes the unit of neighbour   */
/*   t+-1 instead. Emission order: epoch, then k, then thread.              */
/* ------------------------------------------------------------------------ */
uint64_t tg_strided(uint64_t seed, uint32_t n_threads, uint32_t n_epochs, uint32_t per_thread,
                    uint32_t shared_units, double write_p, double redirect_p,
                    uint32_t *ev, uint32_t *counts) {
    static const uint32_t strides[3] = {1u, 2u, 32u};
    sink s = {ev, 0};
    if (counts)
        for (uint32_t t = 0; t < n_threads; t++) counts[t] = n_epochs - 1;
    for (uint32_t e = 0; e < n_epochs; e++) {
        uint32_t st = strides[hsh(seed, 1, e, 0, 0, 0) % 3u];
        for (uint32_t k = 0; k < per_thread; k++) {
            for (uint32_t t = 0; t < n_threads; t++) {
                uint64_t h = hsh(seed, 2, e, k, t, 0);
                uint32_t src = t;
                if (u01(h) < redirect_p) {
                    uint64_t h2 = hsh(seed, 3, e, k, t, 0);
                    src = (h2 & 1u) ? (t + 1u) % n_threads : (t + n_threads - 1u) % n_threads;
                }
                uint32_t unit = (uint32_t)(((uint64_t)src * st + k) % shared_units);
                uint32_t act = (u01(hsh(seed, 4, e, k, t, 0)) < write_p) ? ACT_W : ACT_R;
                emit(&s, unit, 0, t, e, act, SP_SH);
            }
        }
    }
    return s.n;
}

/* ------------------------------------------------------------------------ */
/* Grid of blocks running tree reductions or 32x32 tiled transposes.        */
/* Pattern per block: hash(seed, b) chooses reduction or transpose (50/50). */
/* Global memory: per-block input and output slices of SL units, plus 4096  */
/* counter units at the top that receive atomics. removed_p of the blocks   */
/* lose one barrier k_b (epochs after it are relabelled one lower).         */
/* atomic_p of global reads become atomics on a counter unit; of those,     */
/* peek_p become plain reads of the counter. stray_p of global writes land  */
/* in the next block's output slice or one unit past their own target.     */
/* Emission order: block, epoch, slot, thread.                              */
/* Returns 0 (and emits nothing) when the dimensions do not fit.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    uint32_t n_blocks, block_threads, n_epochs, shared_units, global_units;
    double removed_p, atomic_p, peek_p, stray_p;
} pattern_params;

static uint32_t floor_pow2(uint64_t x) {
    uint32_t p = 1;
    while ((uint64_t)p * 2u <= x && p < 0x80000000u) p *= 2u;
    return p;
}

static uint32_t ilog2u(uint32_t x) { uint32_t l = 0; while ((1u << (l + 1)) <= x) l++; return l; }

/* global read of input slice position pos, possibly turned into a counter atomic/peek */
static inline void global_read(sink *s, const pattern_params *p, uint32_t b, uint32_t t, uint32_t lab,
                               uint32_t in_base, uint32_t sl, uint32_t pos,
                               uint64_t c0, uint64_t c1, uint64_t c2) {
    uint64_t h = hsh(p->seed, 20, c0, c1, c2, t);
    if (u01(h) < p->atomic_p) {
        uint32_t cu = p->global_units - 4096u + (uint32_t)(hsh(p->seed, 21, c0, c1, c2, t) % 4096u);
        uint32_t act = (u01(hsh(p->seed, 22, c0, c1, c2, t)) < p->peek_p) ? ACT_R : ACT_A;
        emit(s, cu, b, t, lab, act, SP_GL);
    } else {
        emit(s, in_base + (pos % sl), b, t, lab, ACT_R, SP_GL);
    }
}

static inline void global_write(sink *s, const pattern_params *p, uint32_t b, uint32_t t, uint32_t lab,
                                uint32_t out0, uint32_t sl, uint32_t pos,
                                uint64_t c0, uint64_t c1, uint64_t c2) {
    uint32_t tb = b;
    const uint64_t h = hsh(p->seed, 23, c0, c1, c2, t);
    if (u01(h) < p->stray_p) {
        /* a stray write: half land in the next block's slice, half one unit over */
        if (hsh(p->seed, 24, c0, c1, c2, t) & 1u) tb = (b + 1u) % p->n_blocks;
        else pos += 1u;
    }
    emit(s, out0 + tb * sl + (pos % sl), b, t, lab, ACT_W, SP_GL);
}

uint64_t tg_pattern(const pattern_params *p, uint32_t *ev, uint32_t *counts) {
    const uint32_t BT = p->block_threads, E = p->n_epochs;
    if (BT < 32 || (BT & (BT - 1)) || BT > 1024 || E < 2 || p->shared_units < 33u * 32u ||
        p->shared_units < BT * 6u + 64u || p->global_units < 4096u + 2u * 1024u * p->n_blocks)
        return 0;
    const uint32_t SL = floor_pow2(((uint64_t)p->global_units - 4096u) / (2ull * p->n_blocks));
    const uint32_t out0 = p->n_blocks * SL;
    const uint32_t L = ilog2u(BT);          /* reduction steps per cycle */
    const uint32_t ROWS = BT / 32u;          /* transpose rows per pass */
    const uint32_t J = (ROWS >= 32u) ? 1u : 32u / ROWS;
    sink s = {ev, 0};

    for (uint32_t b = 0; b < p->n_blocks; b++) {
        const uint64_t hb = hsh(p->seed, 10, b, 0, 0, 0);
        const int transpose = (int)(hb & 1u);
        const int removed = u01(hsh(p->seed, 11, b, 0, 0, 0)) < p->removed_p;
        const uint32_t kb = removed ? (uint32_t)(hsh(p->seed, 12, b, 0, 0, 0) % (E - 1u)) : 0xFFFFFFFFu;
        const uint32_t in_base = b * SL;
        if (counts)
            for (uint32_t t = 0; t < BT; t++) counts[(uint64_t)b * BT + t] = removed ? E - 2u : E - 1u;

        for (uint32_t e = 0; e < E; e++) {
            const uint32_t lab = (removed && e > kb) ? e - 1u : e;
            if (!transpose) {
                /* tree reduction: cycle of L+1 epochs over a double-buffered array
                   sh[base .. base+BT) with base = (cycle & 1) * BT; c==0 loads sh[t]
                   from global, c>=1 halves the active threads: t<s combines sh[t]
                   and sh[t+s]. Consecutive cycles use different halves, so the
                   barrier between them orders nothing. */
                const uint32_t c = e % (L + 1u), y = e / (L + 1u);
                const uint32_t st = (c == 0) ? 0u : (BT >> c);
                const uint32_t base = (y & 1u) * BT;
                for (uint32_t t = 0; t < BT; t++)
                    global_read(&s, p, b, t, lab, in_base, SL, e * BT + t, b, e, 0);
                if (c == 0)
                    for (uint32_t t = 0; t < BT; t++) emit(&s, base + t, b, t, lab, ACT_W, SP_SH);
                else {
                    for (uint32_t t = 0; t < st; t++) emit(&s, base + t, b, t, lab, ACT_R, SP_SH);
                    for (uint32_t t = 0; t < st; t++) emit(&s, base + t + st, b, t, lab, ACT_R, SP_SH);
                    for (uint32_t t = 0; t < st; t++) emit(&s, base + t, b, t, lab, ACT_W, SP_SH);
                }
                /* thread-private scratch: R/W pairs on units no other thread touches */
                for (uint32_t r = 0; r < 2u; r++) {
                    for (uint32_t t = 0; t < BT; t++)
                        emit(&s, 2u * BT + 4u * t + ((e + 2u * r) & 3u), b, t, lab, ACT_R, SP_SH);
                    for (uint32_t t = 0; t < BT; t++)
                        emit(&s, 2u * BT + 4u * t + ((e + 2u * r) & 3u), b, t, lab, ACT_W, SP_SH);
                }
                for (uint32_t t = 0; t < BT; t++)
                    global_read(&s, p, b, t, lab, in_base, SL, e * BT + t + BT / 2u, b, e, 1);
                if (c == L)  /* end of cycle: thread 0 publishes the block partial */
                    global_write(&s, p, b, 0, lab, out0, SL, y, b, e, 2);
            } else {
                /* 32 x ROWS threads move a 32x32 tile (row pitch 33) through shared memory:
                   even epochs read global rows and write tile[r][c];
                   odd epochs read tile[c][r] and write global columns */
                const uint32_t half = e / 2u;
                for (uint32_t j = 0; j < J; j++) {
                    if ((e & 1u) == 0) {
                        for (uint32_t t = 0; t < BT; t++) {
                            const uint32_t tx = t & 31u, ty = t / 32u, r = ty + ROWS * j;
                            if (r >= 32u) continue;
                            global_read(&s, p, b, t, lab, in_base, SL, half * 1024u + r * 32u + tx, b, e, 3u + j);
                        }
                        for (uint32_t t = 0; t < BT; t++) {
                            const uint32_t tx = t & 31u, ty = t / 32u, r = ty + ROWS * j;
                            if (r >= 32u) continue;
                            emit(&s, r * 33u + tx, b, t, lab, ACT_W, SP_SH);
                        }
                    } else {
                        for (uint32_t t = 0; t < BT; t++) {
                            const uint32_t tx = t & 31u, ty = t / 32u, r = ty + ROWS * j;
                            if (r >= 32u) continue;
                            emit(&s, tx * 33u + r, b, t, lab, ACT_R, SP_SH);
                        }
                        for (uint32_t t = 0; t < BT; t++) {
                            const uint32_t tx = t & 31u, ty = t / 32u, r = ty + ROWS * j;
                            if (r >= 32u) continue;
                            global_write(&s, p, b, t, lab, out0, SL, half * 1024u + r * 32u + tx, b, e, 3u + j);
                        }
                    }
                }
            }
        }
    }
    return s.n;
}

/* ------------------------------------------------------------------------ */
/* Barrier-analysis family: shared memory only, per_thread accesses per     */
/* thread per epoch. Epoch e uses region(e) of the shared units (two halves */
/* of size H >= 4*BT); access (t, j) of epoch e touches                      */
/*   region(e)*H + (4t + j + shift(e)) mod (4*BT),  j==0 writes, else reads, */
/* a bijection inside the epoch, so epochs carry no races of their own.     */
/* Barriers in the set `redundant_mask` (bit k = barrier k) switch region,  */
/* so the epochs they separate touch disjoint units; every other barrier    */
/* keeps the region and shifts the mapping by 4099 (3 mod 4), so each write */
/* of epoch k is read by another thread in epoch k+1.                       */
/* redirect_p of accesses move to a random unit of the same region.         */
/* diverge_p of blocks get one thread that skips one barrier: its epochs    */
/* after the skipped barrier are labelled one lower and its count is one    */
/* lower. div_out (optional, n_blocks entries) receives 1 for those blocks.  */
/* Emission order: block, epoch, j, thread.                                 */
/* ------------------------------------------------------------------------ */
uint64_t tg_barrier(uint64_t seed, uint32_t n_blocks, uint32_t block_threads, uint32_t n_epochs,
                    uint32_t shared_units, uint32_t per_thread, uint64_t redundant_mask,
                    double redirect_p, double diverge_p,
                    uint32_t *ev, uint32_t *counts, uint8_t *div_out) {
    const uint32_t BT = block_threads, E = n_epochs, W = 4u * BT;
    if (BT < 2 || BT > 1024 || E < 2 || E > 65 || per_thread < 1 || per_thread > 4 || shared_units < 2u * W)
        return 0;
    const uint32_t H = shared_units / 2u;
    sink s = {ev, 0};
    for (uint32_t b = 0; b < n_blocks; b++) {
        const int div = u01(hsh(seed, 30, b, 0, 0, 0)) < diverge_p;
        const uint32_t td = div ? (uint32_t)(hsh(seed, 31, b, 0, 0, 0) % BT) : 0xFFFFFFFFu;
        const uint32_t kd = div ? (uint32_t)(hsh(seed, 32, b, 0, 0, 0) % (E - 1u)) : 0xFFFFFFFFu;
        if (div_out) div_out[b] = (uint8_t)div;
        if (counts)
            for (uint32_t t = 0; t < BT; t++) counts[(uint64_t)b * BT + t] = (t == td) ? E - 2u : E - 1u;
        uint32_t region = 0, shift = 1u;
        for (uint32_t e = 0; e < E; e++) {
            if (e > 0) {
                if ((redundant_mask >> (e - 1u)) & 1u) region ^= 1u;
                else shift = (shift + 4099u) % W;
            }
            for (uint32_t j = 0; j < per_thread; j++) {
                for (uint32_t t = 0; t < BT; t++) {
                    uint32_t idx = (4u * t + j + shift) % W;
                    if (u01(hsh(seed, 33, b, e, j, t)) < redirect_p)
                        idx = (uint32_t)(hsh(seed, 34, b, e, j, t) % W);
                    const uint32_t lab = (t == td && e > kd) ? e - 1u : e;
                    emit(&s, region * H + idx, b, t, lab, j == 0 ? ACT_W : ACT_R, SP_SH);
                }
            }
        }
    }
    return s.n;
}
