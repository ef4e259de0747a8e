/*
 * ecmc.h -- C ABI of libecmc: event-chain Monte Carlo (ECMC) for hard disks in
 * a periodic square box, many chains at once on one GPU (sm_103a).
 *
 * The method is that of Li, Todo, Maggs & Krauth, "Multithreaded event-chain
 * Monte Carlo with local times" (arXiv:2004.11040): between two breakpoints h
 * and h' = h + ell, k active disks move with v = (1, 0); at a lifting
 * i -> j (Eq. 1) activity passes from the moving disk i to the disk j it
 * touches, and the local time t_j is set to t_i (Sec. 2.1, Alg. 1/2). Each
 * chain advances on its own local time (Sec. 2.2-2.4, Alg. 4-6); the result is
 * that of the global-time process (Alg. 2, Lemma 2).
 *
 * Conventions shared by every call:
 *   - Disks have diameter d (the contact distance; the paper's 2*sigma).
 *   - Positions are FP64 in [0, L). Only x changes during a leg (v = (1,0)).
 *   - Local times are leg-relative: 0 at the start of every leg, ell for the
 *     stalled (still active) disks at its end (Remark 1).
 *   - Chain c owns one active disk; chain order matters only for tie-breaking
 *     of simultaneous events and for the order of the returned lists.
 *   - Every call returns ECMC_OK (0) or a negative ECMC_E* code and never
 *     aborts the process; ecmc_last_error() gives a one-line reason.
 *   - All pointers named "host" are ordinary host memory owned by the caller.
 *     The context owns every device allocation it makes.
 *   - Calls on one context must not run concurrently from several host threads.
 */
#ifndef ECMC_H
#define ECMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ECMC_OK 0
#define ECMC_EINVAL (-1)    /* bad parameters or inputs */
#define ECMC_ENOMEM (-2)    /* device or host allocation failed */
#define ECMC_ECUDA (-3)     /* a CUDA call failed (message in last_error) */
#define ECMC_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define ECMC_ECAPACITY (-5) /* a fixed-size buffer (cell slots, undo log) overflowed */

/* ecmc_params.flags */
#define ECMC_LOG_LIFTINGS 0x1u /* keep every lifting for ecmc_liftings() */
#define ECMC_INPUT_DEVICE 0x2u /* x, y, active passed to ecmc_create are device pointers */
#define ECMC_GRAPH 0x4u        /* find liftings through the constraint graph G(3) (Sec. 3.1)
                                  instead of the cell scan; see "Constraint-graph mode" */
#define ECMC_RESTART 0x8u      /* with ECMC_GRAPH and windows <= 1: conflicts handled by
                                  restart strategy 2 (Sec. 3.4); see "Restart mode" */
#define ECMC_NO_ROWPASS 0x10u  /* cell scan: always use the general parallel pass, also in
                                  windows where the row pass applies (see "Row pass");
                                  results are the same either way */

typedef struct ecmc_ctx ecmc_ctx;

typedef struct {
    int64_t n;              /* number of disks N (>= 3) */
    double box;             /* side L of the periodic square box */
    double d;               /* disk diameter (contact distance), > 0 */
    double ell;             /* chain length between breakpoints (h' - h), > 0 */
    int32_t n_chains;       /* k, 1 <= k <= n */
    int32_t cells_per_side; /* nc; 0 picks the largest nc with L/nc >= d*(1+2^-20).
                               Needs nc >= 3 and L/nc < 1.664*d. */
    uint32_t flags;         /* ECMC_LOG_LIFTINGS | ECMC_INPUT_DEVICE | ECMC_GRAPH |
                               ECMC_RESTART | ECMC_NO_ROWPASS */
    int32_t undo_cap;       /* per-chain event records per leg, < 2^24; 0 = 1024 */
    int64_t log_cap;        /* liftings kept with ECMC_LOG_LIFTINGS; 0 = 1<<22 */
    int32_t windows;        /* claim windows per leg, 1..4096; 0 = 1. A leg is run as W
                               windows of global time [w ell/W, (w+1) ell/W): chains pause
                               (without moving) at a window's end. Results do not depend
                               on W; the conflict flags and the speed do. */
    int32_t reserved;       /* must be 0 */
} ecmc_params;

typedef struct {
    int64_t liftings;        /* liftings (events, Eq. 1) over all legs run */
    int64_t legs;            /* breakpoints reached */
    int64_t conflict_legs;   /* legs in which two chains' scanned cells met */
    int64_t repaired_chains; /* chains in conflict components (once per repair round) */
    int64_t horizon_asserts; /* Eq. 2 failures seen by a conflict-free chain: 0 */
    int64_t order_errors;    /* repaired events found out of time order: 0 */
    double device_ms;        /* device time spent in ecmc_run_to_breakpoint */
    int64_t continued_chains; /* of repaired_chains: in components finished by continuing
                                 the blocked chains (Lemma 2), nothing redone */
    int64_t restarts;         /* ECMC_RESTART: passes begun again at an earlier stop time
                                 T* taken as a breakpoint (Sec. 3.4, strategy 2) */
    int64_t row_windows;      /* claim windows whose parallel pass was the row pass */
    int64_t device_bytes;     /* device memory the context holds (its pooled state) */
    int64_t blocked_chains;   /* chains whose parallel pass stopped at a strong claim of
                                 another chain, summed over windows and legs: the chains
                                 that met another one (Sec. 3.4) */
    int64_t conflict_windows; /* claim windows (legs x W in all) whose conflict flag is 1:
                                 the claim sets of two chains met in the window */
} ecmc_stats_t;

/* One lifting i -> j (Eq. 1): chain c, leg index, time t (= new t_j),
   time of flight tau, x of i at contact, x of j. */
typedef struct {
    int32_t leg, c, i, j;
    double t, tau, xi, xj;
} ecmc_lift_t;

/*
 * ecmc_create -- a context holding the lifted configuration {C_h, A_h}
 * (Sec. 2.1, Alg. 1 input) on the device.
 *   p       problem description (copied).
 *   x, y    n positions each; host pointers unless ECMC_INPUT_DEVICE.
 *           Every coordinate must lie in [0, L); disks must not overlap.
 *   active  k distinct disk ids; chain c starts on active[c].
 *   stream  a cudaStream_t (may be NULL for the default stream) on which all
 *           work of this context is queued; the caller keeps it alive.
 *   out     receives the context; free it with ecmc_destroy.
 * Errors: EINVAL (sizes, ids, coordinates, cell geometry), ENOMEM, ECUDA,
 * ECAPACITY (more disks in a cell than its slots: overlapping input).
 */
int ecmc_create(const ecmc_params *p, const double *x, const double *y,
                const int32_t *active, void *stream, ecmc_ctx **out);

/*
 * ecmc_context_bytes -- the device memory a context created with *p would
 * hold, without allocating anything: its arrays (cells, chain table, event
 * records, claims; with ECMC_GRAPH the disk records, arrows and the graph
 * build's scratch instead of the cells) and the scratch of ecmc_positions,
 * i.e. the device_bytes that ecmc_stats reports once positions have been
 * read. (The persistent launch's scratch, a few kilobytes per system, is not
 * included.) A scheduler admits systems by it. The paper has no counterpart.
 * Errors: EINVAL (bad parameters).
 */
int ecmc_context_bytes(const ecmc_params *p, int64_t *bytes);

/*
 * Constraint-graph mode (ECMC_GRAPH). The context builds, at creation and at
 * every ecmc_set_direction, the constraint graph G(3) of Sec. 3.1: for each
 * disk i and each of three corridors of dy = y_j - y_i (minimum image) --
 * centre |dy| < d/2, upper d/2 <= dy < d, lower -d < dy <= -d/2 -- the disk of
 * least time of flight (tau, then index), or none. While v is fixed disks
 * closer than d in y cannot pass one another, so the arrows stay valid over
 * any number of legs, and a step reads only the (at most three) arrow targets
 * of the active disk. Results (positions, local times, liftings) are those of
 * the cell scan, i.e. of Alg. 2. Claims are taken on the disks a step reads
 * (the active disk and its arrow targets) instead of cells, so a leg's flag
 * is 1 iff in some window the disks that two chains read, each run alone,
 * overlap. Limits: n_chains <= 2^20 - 2. Such contexts are batched with
 * each other only (their own persistent kernel; same claim windows, no
 * ECMC_RESTART). cells_per_side only sets the cell scan that builds the
 * graph.
 *
 * Conflicts. Within a claim window every chain claims, with atomicCAS, each
 * cell it scans; two chains that want one cell "meet". A leg's flag is 1 iff
 * in some window the cells that two chains would scan, each run alone from the
 * window's start, overlap. A cell whose row holds no disk within d in y of the
 * scanning chain's active disk is claimed weakly: it counts for the flag but
 * stops no chain. Chains that met over a cell they read are rolled back and
 * redone in global time order, so results are always those of Alg. 2.
 *
 * ecmc_run_to_breakpoint -- runs n_legs legs of length ell (Alg. 2 semantics:
 * each leg ends at the breakpoint h' with all chains stalled, Remark on
 * stalled spheres), each chain restarting from its stalled disk.
 *   event_budget  0 = run all n_legs; otherwise stop at the first breakpoint
 *                 at which the liftings of this call reach the budget.
 *   leg_flags_out host, n_legs bytes or NULL: the leg's conflict flag (see
 *                 above); entries past *legs_done are untouched.
 *   legs_done     host or NULL: number of legs completed.
 * All legs run in one persistent cooperative launch; returns when they are
 * done (the stream is synchronised).
 * Errors: EINVAL, ECUDA, ECAPACITY (undo log), ETIMEOUT (a grid barrier wait
 * passed its 60 s limit).
 */
int ecmc_run_to_breakpoint(ecmc_ctx *ctx, int32_t n_legs, uint64_t event_budget,
                           uint8_t *leg_flags_out, int32_t *legs_done);

/*
 * ecmc_positions -- copies the current configuration to host arrays: the
 * lifted configuration {C_h, A_h} at the last breakpoint (Sec. 2.1; Alg. 2's
 * output), with the local times of Remark 1 (every disk a chain moved in the
 * last leg carries the time of its last event or stall, measured from the
 * leg's start h, so t_i <= ell):
 *   x, y, t  n doubles each, indexed by disk id (caller-owned; any pointer
 *            may be NULL to skip it); t is leg-relative.
 *   active   k ints: chain c's active (stalled) disk.
 * Synchronises the context's stream. Errors: EINVAL (null ctx), ECUDA.
 */
int ecmc_positions(ecmc_ctx *ctx, double *x, double *y, double *t, int32_t *active);

/*
 * ecmc_set_direction -- direction of motion for the following legs
 * (Sec. 1: in the periodic square box the direction must change at some
 * breakpoints for ECMC to be irreducible; the legs themselves are as in
 * Alg. 2 with v along that direction).
 *   direction  0: +x (the state after ecmc_create); 1: +y.
 * Call between runs (the state is always at a breakpoint then). The context
 * keeps motion along +x of its own frame and is transposed in place (x and y
 * swapped, cells (r, c) <-> (c, r)); ecmc_positions returns x and y in the
 * caller's frame; the xi, xj of ecmc_liftings are along the direction of
 * motion. Local times are reset to 0 (they are leg-relative), and the lifting
 * log is kept. Synchronises the context's stream.
 * Errors: EINVAL (direction not 0 or 1), ECUDA.
 */
int ecmc_set_direction(ecmc_ctx *ctx, int32_t direction);

/*
 * ecmc_set_wait_limit -- bound on every wait of the persistent kernels of the
 * cell-scan path (their grid barriers), in nanoseconds of the device clock;
 * the default, and the largest value, is 60 s. A wait that runs out makes the
 * launch return ECMC_ETIMEOUT (every block stops at its next barrier or
 * gives up waiting for the blocks that stopped), and the context is then in
 * an undefined state: destroy it. A short limit exercises that path; the
 * paper has no counterpart (its threads wait without bound, Sec. 2.3).
 * Errors: EINVAL (ns == 0 or above the default).
 */
int ecmc_set_wait_limit(ecmc_ctx *ctx, uint64_t ns);

/* ecmc_stats -- counters accumulated since ecmc_create, into a host struct
 * owned by the caller: liftings are the events of Eq. 1 (Sec. 2.1; stalls are
 * not events), legs the breakpoints reached (Alg. 2), and the conflict
 * counters read the horizon condition of Eq. 2 as a claim conflict between
 * chains (Sec. 3.4: the violations whose probability grows with the number
 * of chains). Errors: EINVAL (null argument). */
int ecmc_stats(ecmc_ctx *ctx, ecmc_stats_t *out);

/*
 * ecmc_liftings -- the liftings kept under ECMC_LOG_LIFTINGS, leg by leg and,
 * within a leg, chain by chain in the order each chain made them.
 *   buf, cap  caller-owned host array; n_out receives the total count (may
 *             exceed cap; then only cap records are written).
 * Errors: EINVAL if logging was not enabled; ECAPACITY if log_cap overflowed.
 */
int ecmc_liftings(ecmc_ctx *ctx, ecmc_lift_t *buf, int64_t cap, int64_t *n_out);

/*
 * ecmc_graph_arrows -- the constraint graph G(3) of a context created with
 * ECMC_GRAPH (Sec. 3.1), in the context's current frame (motion along +x, or
 * along +y after ecmc_set_direction(ctx, 1), with x and y exchanged):
 *   a  host, 3n int32 or NULL: a[3i + q] = the arrow of disk i in corridor q
 *      (0 centre |dy| < d/2, 1 upper d/2 <= dy < d, 2 lower -d < dy <= -d/2;
 *      dy = y_j - y_i, minimum image), -1 if the corridor holds no disk;
 *   b  host, 3n doubles or NULL: b[3i + q] = sqrt(d^2 - dy^2) of that arrow,
 *      0 where there is none.
 * Both caller-owned. Synchronises the context's stream.
 * Errors: EINVAL (not a graph context), ECUDA.
 */
int ecmc_graph_arrows(ecmc_ctx *ctx, int32_t *a, double *b);

/*
 * ecmc_profile -- device time per phase of the persistent kernel, read from
 * the device clock at the phase boundaries of every ecmc_run_to_breakpoint:
 *   pass1   the parallel pass (one warp per chain, each a task of Alg. 5/6);
 *   repair  component rollback and global-time redo (Alg. 2), with its
 *           union-find rounds;
 *   other   leg start (claims, chain table) and leg end (totals, log).
 * *_launches count legs (pass1, other) and legs with a repair (repair);
 * pass1_liftings counts liftings of the parallel pass (redone ones included),
 * repair_liftings the liftings of legs that needed a repair.
 */
typedef struct {
    int64_t pass1_launches, repair_launches, other_launches;
    int64_t pass1_liftings, repair_liftings;
    double pass1_ms, repair_ms, other_ms;
} ecmc_profile_t;

int ecmc_profile(ecmc_ctx *ctx, ecmc_profile_t *out);

/*
 * Batches: several independent systems (contexts) advanced together by one
 * persistent launch on the device, each leg of each system exactly as
 * ecmc_run_to_breakpoint would compute it (the systems share no state).
 *
 * ecmc_batch_create -- launch scratch for batches, queued on `stream`.
 * ecmc_batch_run    -- runs up to max_legs legs of each of the n_ctx contexts
 *   (distinct; all cell-scan contexts with the same cell slots C and claim
 *   windows, or all constraint-graph contexts with the same claim windows and
 *   without ECMC_RESTART; their streams are synchronised first).
 *   budgets       host, n_ctx liftings or NULL: a context stops at the first
 *                 breakpoint at which its liftings in this call reach its
 *                 budget (0 = no budget); the launch ends when all stopped.
 *   liftings_out, legs_out  host, n_ctx each or NULL: per-context results.
 *   device_ms_out host or NULL: duration of the launch (CUDA events).
 *   Errors: EINVAL, ENOMEM, ECUDA, ECAPACITY, ETIMEOUT (a grid barrier wait
 *   passed its 60 s limit; the launch returned instead of waiting).
 * ecmc_batch_last_error -- reason of the last failure of b.
 * ecmc_batch_destroy    -- releases the scratch to the device memory cache after
 *                         the batch's stream has finished (the contexts stay
 *                         valid).
 */
typedef struct ecmc_batch ecmc_batch;
int ecmc_batch_create(void *stream, ecmc_batch **out);
int ecmc_batch_run(ecmc_batch *b, ecmc_ctx *const *ctxs, int32_t n_ctx, int32_t max_legs,
                   const uint64_t *budgets, int64_t *liftings_out, int32_t *legs_out,
                   double *device_ms_out);
const char *ecmc_batch_last_error(const ecmc_batch *b);
void ecmc_batch_destroy(ecmc_batch *b);

/* ecmc_destroy -- releases every device allocation of ctx (NULL is a no-op)
 * after the work queued on its stream has finished: into the library's device
 * memory cache (below), from which the next context of about the same size
 * takes them. The configuration is lost (read it first with ecmc_positions).
 * The paper's programs keep their state for the whole run; this is the end of
 * a run (Alg. 1 after its last leg). */
void ecmc_destroy(ecmc_ctx *ctx);

/*
 * Device memory cache. Contexts, batches and launches take their device
 * arrays from a process-wide cache, one per device, instead of cudaMalloc, and
 * give them back on destroy instead of cudaFree (each such driver call costs
 * tens to hundreds of microseconds). A request takes the smallest cached block
 * of at least its size and at most an eighth (plus 64 KiB) larger, else a new
 * cudaMalloc; when that fails every cached block is freed and it is tried
 * once more. The paper has no counterpart (its programs allocate once).
 * ecmc_set_cache_limit -- bound on the bytes kept per device (default 4 GiB;
 *   0 keeps nothing): cached blocks beyond it, least recently released
 *   first, are freed at once. Errors: EINVAL (bytes < 0).
 * ecmc_cache_info -- over all devices: the bytes held for reuse, the bytes
 *   handed out and not yet released, and the requests served from the cache
 *   (hits) or by cudaMalloc (misses). Any pointer may be NULL. Never fails.
 */
int ecmc_set_cache_limit(int64_t bytes);
int ecmc_cache_info(int64_t *cached_bytes, int64_t *in_use_bytes, int64_t *hits,
                    int64_t *misses);

/* ecmc_last_error -- reason for the last failure on ctx ("" if none); the
   string belongs to ctx. With ctx == NULL, the last ecmc_create failure. */
const char *ecmc_last_error(const ecmc_ctx *ctx);

/*
 * ecmc_leg_noalloc -- one leg (h -> h + ell), exactly the computation of one
 * leg of ecmc_run_to_breakpoint, for callers that cannot allocate device
 * memory: code running inside a framework whose caching allocator already owns
 * the device heap, real-time loops that may not pay allocation latency, and
 * plug-ins that are handed pointers only. The paper has no counterpart; this
 * is a deployment convenience.
 *
 * The call is synchronous: it returns after the leg has finished on the
 * device (it reads the leg's counters back to decide on the repairs).
 *
 * It allocates nothing (no cudaMalloc, cudaFree or allocating library call, on
 * the device or the host). Its working memory is one file-scope device array
 * of ECMC_NOALLOC_SCRATCH_MIB MiB that the library holds on every GPU that
 * loads it, until the process exits. The first call on a device looks up the
 * array's address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture. Every call shares the array and
 * clears what it needs, so calls that overlap on the GPU (other streams or
 * threads) race and must not be issued.
 *
 *   n, box, d, ell, n_chains, cells_per_side   as in ecmc_params
 *   x        device, n doubles, in/out: positions before and after the leg
 *   y        device, n doubles, in (y never changes for v = (1, 0))
 *   active   device, n_chains ints, in/out: chain c's active disk; on return
 *            its stalled disk, the start disk of the next leg
 *   t_out    device, n doubles, out (NULL to skip): leg-relative local times
 *   stream   cudaStream_t (NULL = default stream); synchronised on return
 *   flag_out host, 1 byte (NULL to skip): 1 if two chains' cells met
 *   lifts_out host (NULL to skip): liftings made in the leg
 * Sizes whose arrays (cells, per-disk and per-chain state, ECMC_NOALLOC_RECORDS
 * event records per chain) do not fit the array return ECMC_EINVAL before any
 * device work; so do bad scalars, coordinates outside [0, L) and repeated or
 * out-of-range active ids. ECMC_ECAPACITY: a chain made more than
 * ECMC_NOALLOC_RECORDS events in the leg, or a cell overflowed. ECMC_ECUDA: a
 * CUDA call failed. Example limits: N = 65536 disks with 256 chains fit.
 */
#define ECMC_NOALLOC_SCRATCH_MIB 24
#define ECMC_NOALLOC_RECORDS 256
int ecmc_leg_noalloc(int64_t n, double box, double d, double ell, int32_t n_chains,
                     int32_t cells_per_side, double *x, const double *y, int32_t *active,
                     double *t_out, void *stream, uint8_t *flag_out, int64_t *lifts_out);

#ifdef __cplusplus
}
#endif

#endif /* ECMC_H */
