/*
 * simulee.h - C ABI of the GB300 synchronization check over simulated
 * memory-access records.
 *
 * The check is the detection half of the memory-model method of Wu et al.,
 * "Characterizing and Detecting CUDA Program Bugs" (arXiv 1905.01833), Sec. 3.2:
 *   - data races          Theorem 1 and Algorithm 5 (Sec. 3.2.3)
 *   - redundant barriers  Algorithm 5 and the definition in Sec. 2
 *   - barrier divergence  Algorithm 4 and the definition in Sec. 2
 * run over a device-resident trace of access records, the Memory Model of
 * Sec. 3.2.1 flattened to one record per access.
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" must point to device memory of the context's
 *     GPU. The report may also be page-locked host memory (cudaHostAlloc or a
 *     pinned torch tensor), which the GPU writes directly.
 *   - The caller owns every buffer: trace, outputs, report and workspace. The
 *     library allocates no device memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream). The return value reports errors the host can see (bad
 *     arguments, workspace too small, a failed launch). Errors found on the
 *     device (a bad record, a wait that gave up, an output cap exceeded) are
 *     written to report->status when the stream reaches them.
 *   - Results are deterministic and identical to the CPU definition: the same
 *     trace gives byte-identical outputs on every run.
 *   - A workspace may be reused by later calls; two calls that share one
 *     workspace must not overlap on the GPU.
 */
#ifndef SIMULEE_H
#define SIMULEE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIMULEE_OK = 0,
    SIMULEE_EINVAL = 1,      /* bad argument or dimensions out of range (host) */
    SIMULEE_EBADTRACE = 2,   /* a record or barrier count is invalid (report) */
    SIMULEE_ENOMEM = 3,      /* workspace too small: below the compact size (host), or a workspace
                                below simulee_workspace_size ran out of stream capacity (report) */
    SIMULEE_ETRUNC = 4,      /* an output held more records than its cap (report) */
    SIMULEE_ETIMEOUT = 5,    /* a bounded device-side wait gave up; outputs unreliable (report) */
    SIMULEE_ECUDA = 6        /* a CUDA call failed (host) */
} simulee_status;

/* actions, spaces, scopes and race classes as stored in records and results */
enum { SIMULEE_READ = 0, SIMULEE_WRITE = 1, SIMULEE_ATOMIC = 2 };
enum { SIMULEE_SHARED = 0, SIMULEE_GLOBAL = 1 };
enum { SIMULEE_INTRA = 0, SIMULEE_INTER = 1 };
enum { SIMULEE_WW = 0, SIMULEE_RW = 1 };

/* trace flags */
#define SIMULEE_FLAG_UNSORTED 1u  /* visit orders need not increase with the record index */
/* Theorem 1's warp refinements (Sec. 3.2.3): the trace carries one statement word per record
   (simulee_trace.stmt), and two accesses of threads in the same warp (same block, same
   tid / 32) race only when both are plain writes of the same statement, or when either was made
   after the warp's threads diverged. Not combinable with SIMULEE_FLAG_UNSORTED. */
#define SIMULEE_FLAG_WARP_AWARE 2u
#define SIMULEE_STMT_DIVERGED 0x80000000u  /* statement-word bit: the access came after divergence */
/* The paper's visit-order counters (Algorithm 3, Sec. 3.2.2): a counter per memory address,
   restarted at 0 for every block (global memory included), bumped by a barrier only when the
   address was visited since its last bump. An access's visit order is then the number of earlier
   epochs in which its block touched its unit, and Algorithm 5 groups by it: intra-block groups are
   unchanged; a barrier k is needed when a unit's accesses in epoch k conflict with its accesses in
   the block's next epoch that touches the unit (empty epochs skipped); global accesses of different
   blocks conflict only at equal visit orders, and such an INTER race record carries that visit
   order in its epoch field. Such traces take the radix-sort path. Not combinable with
   SIMULEE_FLAG_WARP_AWARE. */
#define SIMULEE_FLAG_PAPER_ORDER 4u

/*
 * One access record (16 bytes, four little-endian words): one tuple
 * <visit order, thread, action> of a Memory Unit (Sec. 3.2.1), tagged with its
 * unit, block and barrier epoch.
 *   w[0] unit         4-byte memory unit; < shared_units or < global_units
 *   w[1] visit_order  serial position of the access in the simulated schedule
 *                     (Algorithm 3's round robin); strictly increasing with the
 *                     record index unless SIMULEE_FLAG_UNSORTED
 *   w[2] block        linear block id, < n_blocks
 *   w[3] bits  0..15  tid, linear thread id in the block, < block_threads
 *        bits 16..27  epoch, number of barriers the thread has passed (the
 *                     paper's per-unit visit order, Algorithm 4), <= the
 *                     thread's barrier count
 *        bits 28..29  action (READ, WRITE, ATOMIC; 3 is invalid)
 *        bit  30      space (SHARED: per block; GLOBAL: whole grid)
 *        bit  31      reserved, must be 0
 */
typedef struct { uint32_t w[4]; } simulee_event;

/* A trace. All arrays are device memory owned by the caller. */
typedef struct {
    const simulee_event *events;     /* device, n_events records */
    uint64_t n_events;               /* < 2^31 */
    const uint32_t *barrier_counts;  /* device, n_blocks * block_threads entries: barriers each thread
                                        passed (block-major, then tid) */
    uint32_t n_blocks;               /* >= 1; n_blocks * block_threads <= 2^30 */
    uint32_t block_threads;          /* 1 .. 1024 */
    uint32_t shared_units;           /* shared-memory units per block */
    uint32_t global_units;           /* global-memory units of the grid */
    uint32_t max_barriers;           /* upper bound on every barrier count, <= 4095 */
    uint32_t flags;                  /* SIMULEE_FLAG_* */
    const uint32_t *stmt;            /* with SIMULEE_FLAG_WARP_AWARE: device, n_events statement words
                                        (statement id in bits 0..30 | SIMULEE_STMT_DIVERGED); else NULL */
} simulee_trace;

/*
 * One data race (32 bytes): the lowest conflicting pair of one group and class.
 * A pair conflicts (Theorem 1; its warp conditions only for traces flagged
 * SIMULEE_FLAG_WARP_AWARE) when its owners differ, at least one access writes
 * or is atomic, and not both are atomic.
 * Groups: INTRA = one (space, block, epoch, unit), owners are threads;
 * INTER = one global unit across blocks in any epochs, owners are blocks (with
 * SIMULEE_FLAG_PAPER_ORDER: one global unit and one visit order).
 * Class WW when both accesses modify the unit, RW when one reads.
 * The pair is the one whose later access comes first in schedule order
 * (visit_order, then record index), and among those the earliest partner.
 * INTER records carry block = epoch = 0xFFFFFFFF.
 * Canonical order of the list: (space, scope, block, epoch, unit, cls).
 */
typedef struct {
    uint8_t space, scope, cls, pad;
    uint32_t block, epoch, unit;
    uint32_t vo_first, vo_second;      /* visit orders of the earlier / later access */
    uint32_t gtid_first, gtid_second;  /* block * block_threads + tid of each access */
} simulee_race;

/* A divergent block (Algorithm 4: threads of one block reach different numbers
   of barriers). Listed by block. */
typedef struct { uint32_t block, min_count, max_count, first_min_tid; } simulee_divergence;

/* A redundant barrier (Algorithm 5): barrier k of `block` separates epochs k and
   k+1 and exists when some thread of the block passed it (k < max count). It is
   redundant when merging its two epochs creates no conflicting pair in any unit
   of the block. Barriers are judged one at a time. Listed by (block, barrier). */
typedef struct { uint32_t block, barrier; } simulee_barrier;

/* Output buffers (device). A NULL pointer with cap 0 skips that output's copy
   but its count is still reported. */
typedef struct {
    simulee_race *races;             uint64_t races_cap;
    simulee_divergence *divergence;  uint64_t divergence_cap;
    simulee_barrier *redundant;      uint64_t redundant_cap;
    uint32_t *grid_redundant;        uint64_t grid_redundant_cap;  /* barrier indices redundant in
                                                                       every block that has them */
} simulee_outputs;

/*
 * Per-call report (48 bytes), written by the device. status is OK,
 * EBADTRACE (bad_kind 0: record bad_index; bad_kind 1: barrier_counts entry
 * bad_index; counts are checked before records; outputs untouched and counts
 * 0), ETIMEOUT, ENOMEM (the call's workspace was smaller than
 * simulee_workspace_size and more records needed the radix-sort streams, or
 * more races were staged, than its capacities held; outputs unreliable: call
 * again with simulee_workspace_size bytes), or ETRUNC (some count exceeds its
 * cap; the first cap entries in canonical order were written). n_* are the
 * true counts.
 */
typedef struct {
    int32_t status;
    uint32_t bad_kind;
    uint64_t bad_index;
    uint64_t n_races;
    uint64_t n_divergence;
    uint64_t n_redundant;
    uint64_t n_grid_redundant;
} simulee_report;

typedef enum {
    SIMULEE_PATH_AUTO = 0,  /* per trace: the segment-local hash path where it applies, else sorting */
    SIMULEE_PATH_SORT = 1,  /* always the radix-sort path */
    SIMULEE_PATH_HASH = 2   /* same as AUTO (the hash path still falls back where it cannot apply) */
} simulee_path;

typedef struct {
    uint32_t wait_limit_us;   /* bound on every device-side wait; 0 selects 1,000,000 (1 s) */
    uint32_t path;            /* simulee_path */
    uint32_t test_withhold;   /* testing only: 0 = off; t+1 = tile t of the first sort pass never
                                 publishes its counts, so a later tile's bounded wait gives up */
    uint32_t ingest_ctas_per_sm;   /* persistent CTAs per SM of the record reads; 0 = 2 */
    uint32_t sort_ctas_per_sm;     /* persistent CTAs per SM of each radix pass; 0 = 3 */
    uint32_t reduce_ctas_per_sm;   /* persistent CTAs per SM of the segmented reductions; 0 = 3 */
    uint32_t hash_shape;      /* hash path CTAs: 0 = chosen per call (the smaller shape when blocks have at
                                 most 256 threads and there are at least two blocks per SM), 1 = one 768-thread CTA per SM with
                                 8192-entry run tables (up to 6144 distinct units per run), 2 = two
                                 512-thread CTAs per SM with 4096-entry tables (up to 3072) */
    uint32_t graph_replay;    /* simulee_graph_replay */
    uint32_t sort_items;      /* radix-sort tile: 256 threads x sort_items elements; 0 = 16, or 8 */
    uint32_t radix_bits;      /* digit width of each radix pass: 0 = 8, or 6 or 11 (those widths build
                                 their digit histograms in one extra read of the stream's keys) */
    uint32_t hash_cap_eighths;   /* hash path: a run may hold up to this many eighths of its table in
                                    distinct units before its block goes to the sort path; 0 = 7, or 4..7 */
    uint32_t hash_pool_div;   /* hash path: a run's racy units are resolved in place up to table size /
                                 hash_pool_div of them, beyond that the run goes to the sort path;
                                 0 = 3, or 3..64 */
    uint32_t hot_unit_marks;  /* hash path, block signatures of global units: 0 or 1 = a warp marks a unit
                                 once per run of consecutive lanes that hold the same unit and block, so a
                                 unit that every thread reads (a kernel-wide constant) costs one atomic per
                                 run of lanes rather than one per record; 2 = every record marks (about 2%
                                 less work per record when no unit is that hot) */
    uint32_t hash_groups;     /* hash path, CTAs of the smaller shape (512 threads, 4096-entry tables):
                                 0 = a block whose runs are short (at most 512 or 1024 records per epoch on
                                 average) is checked by a group of 128 or 256 of the CTA's threads with a
                                 quarter or half of its tables, so that a CTA checks four or two such blocks
                                 at once; 1 = every block by a whole CTA */
} simulee_options;

/* Repeated calls. With SIMULEE_GRAPH_AUTO, a check call (simulee_check*, simulee_check_batch,
   simulee_check_noalloc) whose arguments are byte-for-byte those of the previous check call on the
   same context (trace and output descriptors, report, workspace, options; not the device data they
   point to) is issued as one CUDA graph launch: the second such call captures the launch sequence
   (the context keeps one graph) and every later one replays it. The graph reads and writes device
   memory at run time exactly as the direct launches do, so new trace contents in the same buffers
   give new results. Calls on a stream that is being captured, and calls with stage events set, are
   always launched directly. */
typedef enum {
    SIMULEE_GRAPH_AUTO = 0,
    SIMULEE_GRAPH_OFF = 1
} simulee_graph_replay;

typedef struct simulee_ctx simulee_ctx;

/* Create a context on `device` (host object; no device allocation). opt may be NULL. A context
   keeps host state between calls (which kernels are configured, the replay graph of a repeated
   call), so calls on one context must not overlap from several host threads; use one context
   per thread. */
simulee_status simulee_create(simulee_ctx **ctx, int device, const simulee_options *opt);

/* Destroy a context. Pending work on streams is not waited for. */
simulee_status simulee_destroy(simulee_ctx *ctx);

/* Workspace bytes with which simulee_check* never runs out of room for this trace's dimensions and
   size (the worst case: every record through the radix-sort streams, two races per record).
   Only the dimensions, n_events and flags are read (no device access). */
simulee_status simulee_workspace_size(simulee_ctx *ctx, const simulee_trace *trace, size_t *bytes);

/* Compact workspace bytes for a call over n_traces traces (1 for the single-trace entry points).
   The check lays its streams out in whatever workspace it is given: with simulee_workspace_size
   bytes (simulee_batch_workspace_size for a batch) or more it cannot run out of room; with less,
   down to this compact size, its radix-sort streams and race staging get what the workspace holds
   beyond the fixed part. Traces in simulator order take the hash path, which needs those streams
   only for runs it hands over and for the races it finds, so the compact size gives them the
   records of traces that start on the sort path (flags UNSORTED, WARP_AWARE, PAPER_ORDER, or the
   sort path forced in the options) plus max(n/16, 65536) elements. A call that needs more reports
   SIMULEE_ENOMEM in its reports (its outputs are then unreliable) and is repeated with the full
   size. Below this size a call returns SIMULEE_ENOMEM at once (host). No device access. */
simulee_status simulee_compact_workspace_size(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                              size_t *bytes);

/*
 * The whole check in one pass: races (Theorem 1, Algorithm 5), divergence
 * (Algorithm 4) and redundant barriers (Algorithm 5) over one trace.
 * ws: device workspace of at least simulee_compact_workspace_size bytes (simulee_workspace_size
 * bytes never run out of room; see there), 256-byte aligned.
 */
simulee_status simulee_check(simulee_ctx *ctx, const simulee_trace *trace, const simulee_outputs *out,
                             simulee_report *report, void *ws, size_t ws_bytes, void *stream);

/* Races only (Theorem 1; Algorithm 5 race part). report->n_races is the true count. */
simulee_status simulee_check_races(simulee_ctx *ctx, const simulee_trace *trace, simulee_race *out,
                                   uint64_t cap, simulee_report *report, void *ws, size_t ws_bytes,
                                   void *stream);

/* Divergent blocks only (Algorithm 4, Sec. 2). Reads barrier_counts and validates the trace. */
simulee_status simulee_check_divergence(simulee_ctx *ctx, const simulee_trace *trace,
                                        simulee_divergence *out, uint64_t cap, simulee_report *report,
                                        void *ws, size_t ws_bytes, void *stream);

/* Redundant barriers only (Algorithm 5 barrier part). grid may be NULL (grid_cap 0). */
simulee_status simulee_check_redundant_barriers(simulee_ctx *ctx, const simulee_trace *trace,
                                                simulee_barrier *out, uint64_t cap, uint32_t *grid,
                                                uint64_t grid_cap, simulee_report *report, void *ws,
                                                size_t ws_bytes, void *stream);

/*
 * simulee_check_noalloc: the full check (as simulee_check) for callers that
 * cannot allocate device memory: code that runs under a fixed device-memory
 * plan decided at start-up (a server that reserves all GPU memory up front and
 * forbids later allocations), or latency-critical loops where the implicit
 * device synchronisation of cudaMalloc/cudaFree is not acceptable. This entry
 * point allocates nothing: instead of a caller workspace it uses one fixed
 * scratch array of SIMULEE_NOALLOC_SCRATCH_BYTES that the library holds in
 * static device memory; every GPU that loads the library keeps that array until
 * the process exits. The caller still owns and passes the trace, the outputs
 * and the report.
 *   - Size limit: the trace's simulee_workspace_size must not exceed
 *     SIMULEE_NOALLOC_SCRATCH_BYTES; larger traces are rejected with
 *     SIMULEE_ENOMEM before any device work is queued.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current, in the device's primary context); make
 *     that first call before any stream capture is started on that device. A
 *     first call made while `stream` is being captured returns SIMULEE_EINVAL
 *     and queues nothing. If the device's primary context is destroyed and
 *     created again (cudaDeviceReset), the library sees the new context on the
 *     next call and looks the address up again, so that call is again a first
 *     call.
 *   - All calls in the process share the one array (its contents persist from
 *     call to call; each call clears what it needs to start from zero). Calls
 *     that could overlap on the GPU - on different streams, or from different
 *     threads - race on the array: serialise them, e.g. on one stream.
 * The paper has no counterpart of this entry point; it is a deployment aid.
 */
#define SIMULEE_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
simulee_status simulee_check_noalloc(simulee_ctx *ctx, const simulee_trace *trace, const simulee_outputs *out,
                                     simulee_report *report, void *stream);

/*
 * Batched check: n_traces independent traces checked together, each with its
 * own outputs and report (reports: device array of n_traces). Results equal
 * those of checking each trace alone. traces and outs are host arrays read
 * during the call; the trace data they point to is device memory.
 */
simulee_status simulee_batch_workspace_size(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                            size_t *bytes);
simulee_status simulee_check_batch(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                   const simulee_outputs *outs, simulee_report *reports, void *ws,
                                   size_t ws_bytes, void *stream);

/*
 * Fitness of a batch of traces: Eq. 1 of the paper (Sec. 3.3.1, "Intuition")
 * and its secondary fitness R = end - start (Sec. 3.3.2, "Fitness Function"),
 * the scores that guide the evolutionary input generation (Algorithm 1).
 * For memory address i, f(i) = number of distinct threads that access i and
 * g(i) = 1 when i is accessed; F = sum g / sum f (1 when no two threads share
 * an address). An address is a global unit or a shared unit of one block; a
 * thread is block * block_threads + tid; every epoch and action counts.
 * Per trace (out: device array of n_traces, 48 bytes each):
 *   status / bad_kind / bad_index: as in simulee_report (the trace is
 *     validated exactly as by the check; a bad trace reports zero sums);
 *   n_addresses = sum g, n_pairs = sum f (F = n_addresses / n_pairs; a trace
 *     without records has both 0);
 *   shared_lo..hi, global_lo..hi: the accessed unit range of each space
 *     (lo = 0xFFFFFFFF, hi = 0 when the space is not accessed), from which
 *     R = hi - lo of the range the caller's kernel model uses.
 * Limits beyond the check's: the key (trace index, space, block, unit, global
 * thread id) must fit 64 bits (SIMULEE_EINVAL otherwise). traces is a host
 * array read during the call; ws: caller-owned device workspace of at least
 * simulee_fitness_workspace_size bytes, 256-byte aligned. Asynchronous on
 * `stream`.
 */
typedef struct {
    int32_t status;
    uint32_t bad_kind;
    uint64_t bad_index;
    uint64_t n_addresses;
    uint64_t n_pairs;
    uint32_t shared_lo, shared_hi;
    uint32_t global_lo, global_hi;
} simulee_fitness;
simulee_status simulee_fitness_workspace_size(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                              size_t *bytes);
simulee_status simulee_fitness_batch(simulee_ctx *ctx, const simulee_trace *traces, uint32_t n_traces,
                                     simulee_fitness *out, void *ws, size_t ws_bytes, void *stream);

/*
 * Parametric model kernels: the inputs of the evolutionary search for
 * error-inducing launch configurations (Algorithms 1 and 2). Each model
 * stands for a small CUDA kernel; simulee_model_traces writes, for a batch
 * of launch configurations, the traces their simulated executions record
 * (schedule order block, epoch, slot, thread; visit order = serial position
 * within the launch), ready for simulee_fitness_batch and simulee_check.
 *   SIMULEE_MODEL_COPY2D (kaldi's _copy_from_mat of Sec. 2): thread (x, y) of
 *     block (bx, by), X = bx * block_x + x, Y = by * block_y + y, reads global
 *     unit (Y * arg1 + X) mod 2^19 and writes global unit
 *     2^19 + (Y * arg0 + X) mod 2^19; no barrier (barrier counts 0).
 *   SIMULEE_MODEL_STENCIL: 1-D blocks (block_y must be 1); thread t writes
 *     shared unit (t * arg1) mod 4096, passes one barrier, reads shared unit
 *     (t * arg1 + arg0) mod 4096 and writes global unit
 *     (block * block_x + t) mod 2^20 (barrier counts 1).
 * Negative arguments count as 0. Traces use shared_units = 4096 and
 * global_units = 2^20, n_blocks = grid_x * grid_y, block_threads =
 * block_x * block_y (<= 1024). models: device array of n_models, sorted by
 * events_off and by counts_off; launch i writes records
 * [events_off, events_off + threads * (2 or 3)) of events and barrier counts
 * [counts_off, counts_off + threads) of counts (device, caller-owned;
 * n_events / n_counts: their lengths). Asynchronous on `stream`.
 */
enum { SIMULEE_MODEL_COPY2D = 0, SIMULEE_MODEL_STENCIL = 1 };
typedef struct {
    uint32_t model;
    uint32_t grid_x, grid_y, block_x, block_y;
    int32_t arg0, arg1;
    uint32_t reserved;
    uint64_t events_off;
    uint64_t counts_off;
} simulee_model;
simulee_status simulee_model_traces(simulee_ctx *ctx, const simulee_model *models, uint32_t n_models,
                                    simulee_event *events, uint64_t n_events, uint32_t *counts, uint64_t n_counts,
                                    void *stream);

/*
 * Diagnostics.
 * simulee_last_launches: kernels launched by the last check call on this context.
 * simulee_set_stage_events: optional CUDA events (cudaEvent_t, created by the caller
 * with timing enabled) recorded on the call's stream around each stage of the
 * next check calls: events[2*s] before stage s and events[2*s+1] after it, for
 * the stages below (n_events = 2 * SIMULEE_STAGES; NULL / 0 turns recording off).
 * A stage that does not run in a call still records both of its events, back to back.
 */
enum {
    SIMULEE_STAGE_INGEST = 0,   /* count stats; validation and routing of sort-path traces */
    SIMULEE_STAGE_SORT = 1,     /* inter-block filter, radix passes of the record streams */
    SIMULEE_STAGE_REDUCE = 2,   /* segmented reductions: races, epoch adjacency */
    SIMULEE_STAGE_RACES = 3,    /* race filter, canonical race sort and copy-out */
    SIMULEE_STAGE_BLOCKS = 4,   /* divergence, redundant-barrier lists, report */
    SIMULEE_STAGE_HASH = 5,     /* hash path: one read of each block (validation, inter-block stream,
                                   intra-block races, adjacency) */
    SIMULEE_STAGE_FALLBACK = 6, /* routing of what the hash path leaves to the sort path */
    SIMULEE_STAGES = 7
};
uint32_t simulee_last_launches(const simulee_ctx *ctx);
/* 1 when the last check call on this context was issued as one CUDA graph launch (its arguments
   equal the previous call's, graph replay on), 0 when its kernels were launched one by one. */
uint32_t simulee_last_replayed(const simulee_ctx *ctx);
/* Queues on `stream` a copy of five uint32 into dev_out (device memory), for the last check that
   used workspace `ws`: the record counts of the shared-intra, global-intra and global-inter streams
   that went through the radix sort, the number of staged race records, and the number of
   inter-block stream slots written before the inter-block filter (every global record, plus slots
   the hash path reserved and left unused). For measuring algorithmic bytes. */
simulee_status simulee_stream_sizes(simulee_ctx *ctx, const void *ws, uint32_t *dev_out, void *stream);
/* Queues on `stream` a copy of five uint32 into dev_out (device memory), for the last check that
   used workspace `ws`: how the hash path split its blocks into launches. Entries 0..3 are the first
   position of each launch group in the hash path's block list (blocks checked by 128-thread groups
   of the smaller CTAs, by 256-thread groups, by whole smaller CTAs, by the larger CTAs), entry 4 the
   number of blocks listed; group i has entry i+1 - entry i blocks. All zero when no trace took the
   hash path. For measurement and tests. */
simulee_status simulee_hash_groups(simulee_ctx *ctx, const void *ws, uint32_t *dev_out, void *stream);
simulee_status simulee_set_stage_events(simulee_ctx *ctx, void *const *events, uint32_t n_events);

/* Static description of a status code. */
const char *simulee_status_str(simulee_status s);

#ifdef __cplusplus
}
#endif

#endif /* SIMULEE_H */
