/*
 * simulee_oracle.c - CPU ORACLE for the memory-model synchronization check.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke entry point and the
 * benchmark's CPU-baseline leg may load this library. The product path never
 * calls it; it shares no code, header or table with the CUDA library.
 *
 * It is deliberately plain and single threaded: records are grouped with
 * qsort and every group is searched pair by pair, exactly as the definitions
 * read. It follows the paper (Wu et al., "Characterizing and Detecting CUDA
 * Program Bugs", arXiv 1905.01833):
 *   - Memory Model (Sec. 3.2.1): a memory unit holds tuples
 *     <visit order, thread, action>. Here the barrier epoch of a record plays
 *     the role of the paper's per-unit visit order (the count of barriers the
 *     thread has passed), and the record's visit_order field is the serial
 *     position in the simulated schedule, used only to order accesses.
 *   - Theorem 1 (Sec. 3.2.3): two tuples of one unit race when they share the
 *     barrier interval, come from different threads and at least one writes.
 *     The warp refinements of the theorem apply only to traces that carry a
 *     statement word per record (flag WARP_AWARE, orc_check2): two accesses
 *     of threads in the same warp then race only when both are plain writes
 *     of the same statement, or when either was made after the warp's
 *     threads diverged. Otherwise they are not applied. Atomics count as
 *     writes except that two atomics never race; global memory is also
 *     checked across blocks, where barriers give no order, in any epochs.
 *   - Algorithm 5 (Sec. 3.2.3): races per unit and visit-order group; a
 *     barrier is redundant when merging the tuples of the two visit orders it
 *     separates creates no race.
 *   - Algorithm 4 and Sec. 2 (barrier divergence): threads of one block that
 *     reach different numbers of barriers.
 *   - Paper visit orders (flag PAPER_ORDER): Algorithm 3 keeps one visit-order
 *     counter per memory address, set to 0 for every block (for global memory
 *     too), and a barrier bumps an address's counter only if the address was
 *     visited since its last bump. An access's visit order is then the number
 *     of earlier epochs in which its block touched its unit (the unit's
 *     non-empty epochs, counted). Algorithm 5 groups a unit's tuples by visit
 *     order: inside a block that is the same as grouping by epoch, but the
 *     tuples of a global unit from different blocks now meet only at equal
 *     visit orders, and a barrier's adjacent groups are a unit's accesses
 *     before it and at the unit's next non-empty epoch of the block.
 * Output conventions (one record per group and class, the lowest pair, the
 * canonical order) are the ones this library defines; see the header of the
 * Python wrapper for the full statement.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EBADTRACE 2
#define ORC_ENOMEM 3

#define ACT_R 0u
#define ACT_W 1u
#define ACT_A 2u

#define FLAG_UNSORTED 1u
#define FLAG_WARP_AWARE 2u
#define FLAG_PAPER_ORDER 4u
#define STMT_DIVERGED 0x80000000u

typedef struct {
    uint8_t space, scope, cls, pad;
    uint32_t block, epoch, unit, vo_first, vo_second, gtid_first, gtid_second;
} orc_race;                                               /* 32 bytes */

typedef struct { uint32_t block, min_count, max_count, first_min_tid; } orc_div;
typedef struct { uint32_t block, barrier; } orc_bar;

typedef struct {
    int32_t status;
    uint32_t bad_kind;          /* 0: a record, 1: a barrier count */
    uint64_t bad_index;
    orc_race *races; uint64_t n_races;
    orc_div *divs; uint64_t n_divs;
    orc_bar *bars; uint64_t n_bars;
    uint32_t *grid; uint64_t n_grid;
} orc_result;

typedef struct {                 /* one decoded record */
    uint32_t unit, vo, block, tid, epoch, act, space, gtid;
    uint32_t stmt;               /* statement id | STMT_DIVERGED (warp-aware traces) */
    uint32_t wa;                 /* the trace is warp-aware */
    uint32_t rank;               /* PAPER_ORDER: earlier non-empty epochs of (space, block, unit) */
} rec_t;

typedef struct { uint64_t k0, k1, k2, idx; } skey;

static int cmp_skey(const void *a, const void *b) {
    const skey *x = (const skey *)a, *y = (const skey *)b;
    if (x->k0 != y->k0) return x->k0 < y->k0 ? -1 : 1;
    if (x->k1 != y->k1) return x->k1 < y->k1 ? -1 : 1;
    if (x->k2 != y->k2) return x->k2 < y->k2 ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* write or atomic: the actions that modify the unit */
static int modifies(uint32_t act) { return act == ACT_W || act == ACT_A; }

/* Theorem 1 plus the atomic rule: different owners, at least one modifying
   access, not both atomic. For warp-aware traces, two threads of one warp
   (same block, same tid / 32) race only when both plainly write by the same
   statement, or when either access came after the warp diverged. */
static int same_warp(const rec_t *p, const rec_t *q) {
    return p->block == q->block && (p->tid >> 5) == (q->tid >> 5);
}
static int conflict(const rec_t *p, const rec_t *q, uint32_t id_p, uint32_t id_q) {
    if (id_p == id_q) return 0;
    if (!modifies(p->act) && !modifies(q->act)) return 0;
    if (p->act == ACT_A && q->act == ACT_A) return 0;
    if (p->wa && same_warp(p, q)) {
        const int same_statement_writes = p->act == ACT_W && q->act == ACT_W &&
                                          (p->stmt & ~STMT_DIVERGED) == (q->stmt & ~STMT_DIVERGED);
        const int diverged = (p->stmt & STMT_DIVERGED) || (q->stmt & STMT_DIVERGED);
        if (!same_statement_writes && !diverged) return 0;
    }
    return 1;
}

/* class of a conflicting pair: 0 = write&write, 1 = read&write */
static uint32_t pair_class(const rec_t *p, const rec_t *q) {
    return (modifies(p->act) && modifies(q->act)) ? 0u : 1u;
}

static void orc_free_fields(orc_result *r) {
    free(r->races); free(r->divs); free(r->bars); free(r->grid);
    r->races = NULL; r->divs = NULL; r->bars = NULL; r->grid = NULL;
}

void orc_free(orc_result *r) {
    if (!r) return;
    orc_free_fields(r);
    free(r);
}

/* ---- validation ------------------------------------------------------------ */
static int validate(const uint32_t *ev, uint64_t n, const uint32_t *counts, uint32_t nb, uint32_t bt,
                    uint32_t su, uint32_t gu, uint32_t maxb, uint32_t flags,
                    uint32_t *bad_kind, uint64_t *bad_index) {
    uint64_t nt = (uint64_t)nb * bt;
    for (uint64_t i = 0; i < nt; i++) {
        if (counts[i] > maxb) { *bad_kind = 1; *bad_index = i; return 1; }
    }
    for (uint64_t i = 0; i < n; i++) {
        const uint32_t *w = ev + 4 * i;
        uint32_t unit = w[0], vo = w[1], block = w[2], w3 = w[3];
        uint32_t tid = w3 & 0xFFFFu, epoch = (w3 >> 16) & 0xFFFu, act = (w3 >> 28) & 3u;
        uint32_t space = (w3 >> 30) & 1u, reserved = w3 >> 31;
        int bad = 0;
        if (block >= nb || tid >= bt) bad = 1;
        if (act == 3u || reserved) bad = 1;
        if (space == 0 && unit >= su) bad = 1;
        if (space == 1 && unit >= gu) bad = 1;
        if (!bad && epoch > counts[(uint64_t)block * bt + tid]) bad = 1;
        if (!(flags & FLAG_UNSORTED) && i > 0 && vo <= ev[4 * (i - 1) + 1]) bad = 1;
        if (bad) { *bad_kind = 0; *bad_index = i; return 1; }
    }
    return 0;
}

static void decode(const uint32_t *ev, uint64_t n, uint32_t bt, const uint32_t *stmt, rec_t *r) {
    for (uint64_t i = 0; i < n; i++) {
        r[i].stmt = stmt ? stmt[i] : 0u;
        r[i].wa = stmt ? 1u : 0u;
        r[i].rank = 0;
        const uint32_t *w = ev + 4 * i;
        r[i].unit = w[0];
        r[i].vo = w[1];
        r[i].block = w[2];
        r[i].tid = w[3] & 0xFFFFu;
        r[i].epoch = (w[3] >> 16) & 0xFFFu;
        r[i].act = (w[3] >> 28) & 3u;
        r[i].space = (w[3] >> 30) & 1u;
        r[i].gtid = w[2] * bt + r[i].tid;
    }
}

/* ---- growable output arrays ------------------------------------------------- */
typedef struct { void *p; uint64_t n, cap; size_t sz; } vec;
static int vec_push(vec *v, const void *item) {
    if (v->n == v->cap) {
        uint64_t nc = v->cap ? v->cap * 2 : 64;
        void *np_ = realloc(v->p, nc * v->sz);
        if (!np_) return 0;
        v->p = np_; v->cap = nc;
    }
    memcpy((char *)v->p + v->n * v->sz, item, v->sz);
    v->n++;
    return 1;
}

/*
 * Lowest conflicting pair of class `cls` in a group whose records are listed
 * in schedule order (visit order, then record index). "Lowest" means the pair
 * whose later access comes first; among those, the earliest partner. The
 * search is the definition itself: scan q in order and, for each q, the
 * partners before it in order; the first hit is the answer.
 * inter != 0: owners are blocks, else global thread ids.
 */
static int lowest_pair(const rec_t *r, const skey *g, uint64_t m, uint32_t cls, int inter,
                       uint64_t *pi, uint64_t *qi) {
    for (uint64_t q = 1; q < m; q++) {
        const rec_t *rq = &r[g[q].idx];
        uint32_t idq = inter ? rq->block : rq->gtid;
        for (uint64_t p = 0; p < q; p++) {
            const rec_t *rp = &r[g[p].idx];
            uint32_t idp = inter ? rp->block : rp->gtid;
            if (conflict(rp, rq, idp, idq) && pair_class(rp, rq) == cls) {
                *pi = g[p].idx; *qi = g[q].idx;
                return 1;
            }
        }
    }
    return 0;
}

/* a group can only race if it holds a write, or an atomic next to a non-atomic */
static int may_race(const rec_t *r, const skey *g, uint64_t m) {
    int has_w = 0, has_a = 0, has_r = 0;
    for (uint64_t i = 0; i < m; i++) {
        uint32_t a = r[g[i].idx].act;
        has_w |= (a == ACT_W); has_a |= (a == ACT_A); has_r |= (a == ACT_R);
    }
    return has_w || (has_a && has_r);
}

static int emit_group(vec *out, const rec_t *r, const skey *g, uint64_t m, int inter, int paper) {
    if (m < 2 || !may_race(r, g, m)) return 1;
    for (uint32_t cls = 0; cls < 2; cls++) {
        uint64_t pi, qi;
        if (!lowest_pair(r, g, m, cls, inter, &pi, &qi)) continue;
        const rec_t *p = &r[pi], *q = &r[qi];
        orc_race x;
        memset(&x, 0, sizeof x);
        x.space = (uint8_t)q->space;
        x.scope = (uint8_t)(inter ? 1 : 0);
        x.cls = (uint8_t)cls;
        x.block = inter ? 0xFFFFFFFFu : q->block;
        x.epoch = inter ? (paper ? q->rank : 0xFFFFFFFFu) : q->epoch;
        x.unit = q->unit;
        x.vo_first = p->vo; x.vo_second = q->vo;
        x.gtid_first = p->gtid; x.gtid_second = q->gtid;
        if (!vec_push(out, &x)) return 0;
    }
    return 1;
}

/* ---- paper visit orders: per (space, block, unit), the number of distinct earlier epochs --- */
static int paper_ranks(rec_t *r, uint64_t n) {
    skey *k = (skey *)malloc((n ? n : 1) * sizeof(skey));
    if (!k) return 0;
    for (uint64_t i = 0; i < n; i++) {
        k[i].k0 = ((uint64_t)r[i].space << 32) | r[i].block;
        k[i].k1 = ((uint64_t)r[i].unit << 32) | r[i].epoch;
        k[i].k2 = 0;
        k[i].idx = i;
    }
    qsort(k, n, sizeof(skey), cmp_skey);
    uint32_t rank = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (i == 0 || k[i].k0 != k[i - 1].k0 || (k[i].k1 >> 32) != (k[i - 1].k1 >> 32)) rank = 0;
        else if (k[i].k1 != k[i - 1].k1) rank++;
        r[k[i].idx].rank = rank;
    }
    free(k);
    return 1;
}

/* ---- races: intra-block groups (space, block, epoch, unit), then inter-block
        groups (global unit); emitted in canonical order ---------------------- */
static int races(const rec_t *r, uint64_t n, int paper, vec *out) {
    skey *k = (skey *)malloc((n ? n : 1) * sizeof(skey));
    if (!k) return 0;
    for (uint64_t i = 0; i < n; i++) {
        k[i].k0 = ((uint64_t)r[i].space << 32) | r[i].block;
        k[i].k1 = ((uint64_t)r[i].epoch << 32) | r[i].unit;
        k[i].k2 = r[i].vo;
        k[i].idx = i;
    }
    qsort(k, n, sizeof(skey), cmp_skey);
    for (uint64_t s = 0; s < n;) {
        uint64_t e = s + 1;
        while (e < n && k[e].k0 == k[s].k0 && k[e].k1 == k[s].k1) e++;
        if (!emit_group(out, r, k + s, e - s, 0, paper)) { free(k); return 0; }
        s = e;
    }
    /* inter-block: global records grouped by unit only (paper visit orders: by visit order, then unit,
       which is also the canonical order of the records emitted) */
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (r[i].space != 1) continue;
        k[m].k0 = paper ? r[i].rank : r[i].unit; k[m].k1 = paper ? r[i].unit : 0; k[m].k2 = r[i].vo; k[m].idx = i;
        m++;
    }
    qsort(k, m, sizeof(skey), cmp_skey);
    for (uint64_t s = 0; s < m;) {
        uint64_t e = s + 1;
        while (e < m && k[e].k0 == k[s].k0 && k[e].k1 == k[s].k1) e++;
        if (!emit_group(out, r, k + s, e - s, 1, paper)) { free(k); return 0; }
        s = e;
    }
    free(k);
    return 1;
}

/* ---- redundant barriers ------------------------------------------------------
   Barrier k of block b separates epochs k and k+1. It is NOT redundant iff some
   unit (either space) of block b has a record p of epoch k and a record q of
   epoch k+1 that would race if the two epochs were one (owners: threads).
   Paper visit orders: q is in the unit's next non-empty epoch of block b after
   k (the group of the next visit order), whichever epoch that is. */
static int barriers(const rec_t *r, uint64_t n, const uint32_t *counts, uint32_t nb, uint32_t bt,
                    uint32_t maxb, int paper, vec *bars, vec *grid) {
    uint64_t ne = (uint64_t)maxb + 1;
    uint8_t *nonred = (uint8_t *)calloc((uint64_t)nb * ne + 1, 1);
    uint32_t *maxc = (uint32_t *)calloc((uint64_t)nb + 1, sizeof(uint32_t));
    skey *k = (skey *)malloc((n ? n : 1) * sizeof(skey));
    if (!nonred || !maxc || !k) { free(nonred); free(maxc); free(k); return 0; }
    for (uint32_t b = 0; b < nb; b++)
        for (uint32_t t = 0; t < bt; t++)
            if (counts[(uint64_t)b * bt + t] > maxc[b]) maxc[b] = counts[(uint64_t)b * bt + t];
    for (uint64_t i = 0; i < n; i++) {
        k[i].k0 = ((uint64_t)r[i].space << 32) | r[i].block;
        k[i].k1 = ((uint64_t)r[i].unit << 32) | r[i].epoch;
        k[i].k2 = r[i].vo;
        k[i].idx = i;
    }
    qsort(k, n, sizeof(skey), cmp_skey);
    for (uint64_t s = 0; s < n;) {           /* one (space, block, unit, epoch) group at a time */
        uint64_t e = s + 1;
        while (e < n && k[e].k0 == k[s].k0 && k[e].k1 == k[s].k1) e++;
        /* the next group: same (space, block, unit), epoch + 1 (paper visit orders: any later epoch) ? */
        if (e < n && k[e].k0 == k[s].k0 && (k[e].k1 >> 32) == (k[s].k1 >> 32) &&
            (paper || (k[e].k1 & 0xFFFFFFFFu) == (k[s].k1 & 0xFFFFFFFFu) + 1)) {
            uint64_t f = e + 1;
            while (f < n && k[f].k0 == k[e].k0 && k[f].k1 == k[e].k1) f++;
            const rec_t *r0 = &r[k[s].idx];
            uint64_t slot = (uint64_t)r0->block * ne + r0->epoch;
            for (uint64_t i = s; i < e && !nonred[slot]; i++)
                for (uint64_t j = e; j < f; j++) {
                    const rec_t *p = &r[k[i].idx], *q = &r[k[j].idx];
                    if (conflict(p, q, p->gtid, q->gtid)) { nonred[slot] = 1; break; }
                }
        }
        s = e;
    }
    uint32_t gmax = 0;
    for (uint32_t b = 0; b < nb; b++) {
        if (maxc[b] > gmax) gmax = maxc[b];
        for (uint32_t kk = 0; kk < maxc[b]; kk++)
            if (!nonred[(uint64_t)b * ne + kk]) {
                orc_bar x = {b, kk};
                if (!vec_push(bars, &x)) goto fail;
            }
    }
    /* grid-wide: barrier k is redundant in every block that has it */
    for (uint32_t kk = 0; kk < gmax; kk++) {
        int all = 1;
        for (uint32_t b = 0; b < nb && all; b++)
            if (maxc[b] > kk && nonred[(uint64_t)b * ne + kk]) all = 0;
        if (all && !vec_push(grid, &kk)) goto fail;
    }
    free(nonred); free(maxc); free(k);
    return 1;
fail:
    free(nonred); free(maxc); free(k);
    return 0;
}

/* ---- barrier divergence: a block whose threads reach unequal barrier counts --- */
static int divergence(const uint32_t *counts, uint32_t nb, uint32_t bt, vec *out) {
    for (uint32_t b = 0; b < nb; b++) {
        uint32_t mn = 0xFFFFFFFFu, mx = 0, first = 0;
        for (uint32_t t = 0; t < bt; t++) {
            uint32_t c = counts[(uint64_t)b * bt + t];
            if (c < mn) { mn = c; first = t; }
            if (c > mx) mx = c;
        }
        if (bt > 0 && mn != mx) {
            orc_div x = {b, mn, mx, first};
            if (!vec_push(out, &x)) return 0;
        }
    }
    return 1;
}

/*
 * Full check. ev: n records of 4 uint32 words; counts: nb*bt per-thread barrier
 * counts. Returns a heap result (free with orc_free), or NULL when out of memory.
 */
orc_result *orc_check2(const uint32_t *ev, uint64_t n, const uint32_t *counts, uint32_t nb, uint32_t bt,
                       uint32_t su, uint32_t gu, uint32_t maxb, uint32_t flags, const uint32_t *stmt) {
    orc_result *res = (orc_result *)calloc(1, sizeof(orc_result));
    if (!res) return NULL;
    if (validate(ev, n, counts, nb, bt, su, gu, maxb, flags, &res->bad_kind, &res->bad_index)) {
        res->status = ORC_EBADTRACE;
        return res;
    }
    rec_t *r = (rec_t *)malloc((n ? n : 1) * sizeof(rec_t));
    if (!r) { free(res); return NULL; }
    decode(ev, n, bt, (flags & FLAG_WARP_AWARE) ? stmt : NULL, r);
    const int paper = (flags & FLAG_PAPER_ORDER) != 0;
    vec rv = {0, 0, 0, sizeof(orc_race)}, dv = {0, 0, 0, sizeof(orc_div)};
    vec bv = {0, 0, 0, sizeof(orc_bar)}, gv = {0, 0, 0, sizeof(uint32_t)};
    int ok = (!paper || paper_ranks(r, n)) && races(r, n, paper, &rv) && divergence(counts, nb, bt, &dv) &&
             barriers(r, n, counts, nb, bt, maxb, paper, &bv, &gv);
    free(r);
    res->races = (orc_race *)rv.p; res->n_races = rv.n;
    res->divs = (orc_div *)dv.p; res->n_divs = dv.n;
    res->bars = (orc_bar *)bv.p; res->n_bars = bv.n;
    res->grid = (uint32_t *)gv.p; res->n_grid = gv.n;
    if (!ok) { orc_free(res); return NULL; }
    res->status = ORC_OK;
    return res;
}

/* ---- fitness (Sec. 3.3.1, Eq. 1) --------------------------------------------
 * For memory address i: f(i) = the number of distinct threads that access i,
 * g(i) = 1 when some thread accesses i. Eq. 1's fitness is sum g / sum f. An
 * address is a global unit (one for the whole grid) or a shared unit of one
 * block; a thread is its global id block * block_threads + tid; all epochs and
 * actions count. Also returned: the accessed unit range [lo, hi] of each space
 * (the secondary fitness R = end - start; lo = 0xFFFFFFFF, hi = 0 when the
 * space is not accessed). The trace is validated exactly as by orc_check.
 * Written out directly: sort the (space, block or 0, unit, gtid) tuples, count
 * distinct tuples and distinct (space, block or 0, unit) prefixes. */
typedef struct { uint32_t space, block, unit, gtid; } ftuple;

static int cmp_ftuple(const void *a, const void *b) {
    const ftuple *x = (const ftuple *)a, *y = (const ftuple *)b;
    if (x->space != y->space) return x->space < y->space ? -1 : 1;
    if (x->block != y->block) return x->block < y->block ? -1 : 1;
    if (x->unit != y->unit) return x->unit < y->unit ? -1 : 1;
    if (x->gtid != y->gtid) return x->gtid < y->gtid ? -1 : 1;
    return 0;
}

/* Returns ORC_OK, ORC_EBADTRACE (bad_kind / bad_index set) or ORC_ENOMEM.
 * out6 = {n_addresses, n_pairs} as uint64; range4 = {shared lo, shared hi, global lo, global hi}. */
int32_t orc_fitness(const uint32_t *ev, uint64_t n, const uint32_t *counts, uint32_t nb, uint32_t bt,
                    uint32_t su, uint32_t gu, uint32_t maxb, uint32_t flags, uint32_t *bad_kind,
                    uint64_t *bad_index, uint64_t *n_addresses, uint64_t *n_pairs, uint32_t *range4) {
    *bad_kind = 0;
    *bad_index = 0;
    *n_addresses = 0;
    *n_pairs = 0;
    range4[0] = range4[2] = 0xFFFFFFFFu;
    range4[1] = range4[3] = 0;
    if (validate(ev, n, counts, nb, bt, su, gu, maxb, flags, bad_kind, bad_index)) return ORC_EBADTRACE;
    ftuple *t = (ftuple *)malloc((n ? n : 1) * sizeof(ftuple));
    if (!t) return ORC_ENOMEM;
    for (uint64_t i = 0; i < n; i++) {
        const uint32_t *w = ev + 4 * i;
        const uint32_t space = (w[3] >> 30) & 1u, unit = w[0], block = w[2], tid = w[3] & 0xFFFFu;
        t[i].space = space;
        t[i].block = space ? 0u : block;
        t[i].unit = unit;
        t[i].gtid = block * bt + tid;
        uint32_t *lo = &range4[2 * space], *hi = &range4[2 * space + 1];
        if (unit < *lo) *lo = unit;
        if (unit > *hi) *hi = unit;
    }
    qsort(t, n, sizeof(ftuple), cmp_ftuple);
    for (uint64_t i = 0; i < n; i++) {
        const int new_pair = i == 0 || cmp_ftuple(&t[i - 1], &t[i]) != 0;
        const int new_addr = i == 0 || t[i - 1].space != t[i].space || t[i - 1].block != t[i].block ||
                             t[i - 1].unit != t[i].unit;
        *n_pairs += (uint64_t)new_pair;
        *n_addresses += (uint64_t)new_addr;
    }
    free(t);
    return ORC_OK;
}

/* The check without statement words (warp refinements off). */
orc_result *orc_check(const uint32_t *ev, uint64_t n, const uint32_t *counts, uint32_t nb, uint32_t bt,
                      uint32_t su, uint32_t gu, uint32_t maxb, uint32_t flags) {
    return orc_check2(ev, n, counts, nb, bt, su, gu, maxb, flags & ~FLAG_WARP_AWARE, NULL);
}

/* flat accessors for foreign-function callers */
int32_t orc_status(const orc_result *r) { return r->status; }
uint32_t orc_bad_kind(const orc_result *r) { return r->bad_kind; }
uint64_t orc_bad_index(const orc_result *r) { return r->bad_index; }
uint64_t orc_n_races(const orc_result *r) { return r->n_races; }
uint64_t orc_n_divs(const orc_result *r) { return r->n_divs; }
uint64_t orc_n_bars(const orc_result *r) { return r->n_bars; }
uint64_t orc_n_grid(const orc_result *r) { return r->n_grid; }
void orc_copy(const orc_result *r, void *races, void *divs, void *bars, void *grid) {
    if (races && r->n_races) memcpy(races, r->races, r->n_races * sizeof(orc_race));
    if (divs && r->n_divs) memcpy(divs, r->divs, r->n_divs * sizeof(orc_div));
    if (bars && r->n_bars) memcpy(bars, r->bars, r->n_bars * sizeof(orc_bar));
    if (grid && r->n_grid) memcpy(grid, r->grid, r->n_grid * sizeof(uint32_t));
}
