/*
 * ecmc_oracle.c -- plain, slow CPU oracle for event-chain Monte Carlo (ECMC)
 * of two-dimensional hard disks between two breakpoints, after Li, Todo,
 * Maggs & Krauth, "Multithreaded event-chain Monte Carlo with local times"
 * (arXiv:2004.11040).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file. The CUDA path shares no code, header,
 * table or helper with it. Compile with -O2 -ffp-contract=off -fno-fast-math
 * so that every double operation below is one IEEE-754 round-to-nearest
 * operation in the order written.
 *
 * What it computes (all in FP64):
 *   orc_leg      -- Alg. 2 (ECMC with global time) from a lifted configuration
 *                   {C_h, A_h} to the next breakpoint h' = h + ell, with
 *                   v = (1, 0). Events are taken in order of their global time
 *                   T (ties: lower chain index first). Output: C_{h'}, A_{h'},
 *                   the local times and the set of liftings (Eq. 1).
 *                   It also returns the leg's conflict flag. The leg is cut
 *                   into W windows of global time, [w ell/W, (w+1) ell/W);
 *                   at the start of each window every unfinished chain is run
 *                   alone from the current state (Alg. 4 with a single chain,
 *                   the other chains' disks counted as static) through its
 *                   events before the window's end, while the cells it scans
 *                   are recorded; the flag is 1 iff in some window one cell
 *                   is scanned by two chains. The windows only decide the
 *                   flag: the events executed are those of Alg. 2 whatever W.
 *   orc_alg4_leg -- Alg. 4 (single-threaded ECMC with local times): chains
 *                   run one after another on the shared state, the horizon
 *                   condition (Eq. 2, strict: t_i + tau_ij > t_j, as Alg. 5
 *                   tests it) is checked for every candidate, and a chain that
 *                   would lift onto an active disk moves up to contact and
 *                   stops (Remark 10). Lemma 2: without a violation its output
 *                   equals that of orc_leg.
 *
 * Readings of the paper used here (each one a choice the paper leaves open):
 *   - Time of flight (Sec. 2.2, Eq. 2; Alg. 5; Eq. 3 in Sec. 3.1):
 *     tau_ij = dx - b_ij with b_ij = sqrt(d^2 - dy^2). The printed "+ b_ij"
 *     in the text after Eq. 2 contradicts the time of flight that Alg. 5
 *     computes and the contact inequality of Eq. 3; the minus sign is used.
 *   - Periodic box (Sec. 1 says contact "must be adapted"): dx is the forward
 *     image x_j - x_i (+L if negative); dy is the minimum image; j is a
 *     candidate iff dy < d (strict, Sec. 3.1 corridors); tau is clamped at 0
 *     (absorbs rounding left by an earlier contact); x is kept in [0, L).
 *   - Ties (Sec. 1 says liftings are generically at distinct times): the
 *     target is the argmin of (tau, j) over candidates; a lift happens iff
 *     tau* < D (the remaining chain length reaches the contact), otherwise
 *     the chain moves by D and stalls at the breakpoint.
 *     Events with equal global time run in chain order.
 *   - Active and stalled disks of other chains are not candidates in Alg. 2
 *     (the minimum runs over i in A, j not in A).
 *   - Local times are leg-relative (h = 0): t_i and the remaining distance D
 *     are updated separately, t_j then t_i then x_i (Remark 11: the local
 *     time is set before the position moves).
 *   - Cell scan (the paper gives none): cells of side a = L/nc (a > d),
 *     cell(v) = (int)(v * (nc/L)) clamped to nc-1; rows cy-1..cy+1; columns
 *     cx, cx+1, ... ; before column m >= 1 the scan stops if
 *     (m*a - fx) - d > best + eps with best = min(D, best candidate tau),
 *     fx = x_i - cx*a and eps = L * 2^-30. The margin makes the cell scan
 *     return the same lifting as the all-pairs definition (tested).
 *   - An "event" is a lifting i -> j; stalls are not events.
 *   - Constraint graph G(3) (Sec. 3.1): the arrows of disk i are, in each of
 *     three corridors of the minimum-image dy = y_j - y_i -- centre
 *     |dy| < d/2, upper d/2 <= dy < d, lower -d < dy <= -d/2 -- the disk of
 *     least (tau_ij, j) with tau as above (all local times 0: the graph is
 *     taken from a synchronised configuration, the start of a leg), or none
 *     if the corridor is empty. Disks closer than d in y cannot pass one
 *     another under v = (1, 0), so the arrows hold for as long as v does.
 *     With search == 2 every step takes its candidates from the arrows of the
 *     active disk alone, and the conflict flag is computed from the disks a
 *     step reads (the active disk and its arrow targets) instead of cells.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TAG_STATIC 0
#define TAG_ACTIVE 1
#define TAG_STALLED 2

typedef struct {
    int32_t leg, c, i, j;
    double t;   /* lifting time = new local time of j */
    double tau; /* time of flight */
    double xi;  /* x of i at contact */
    double xj;  /* x of j */
} orc_lift;

/* Shared problem description. Arrays are owned by the caller. */
typedef struct {
    int64_t n;
    double L, d, ell;
    int32_t nc;      /* cells per side (scan and claims) */
    int32_t search;  /* 0: all pairs (definition), 1: cell scan, 2: constraint graph */
    int32_t windows; /* claim windows per leg (>= 1), see orc_leg */
    int32_t pad;
} orc_params;

/* ------------------------------------------------------------------ geometry */

static double fwd_dx(double xj, double xi, double L) {
    double dx = xj - xi;
    if (dx < 0.0) dx += L;
    return dx;
}

static double perp_dist(double yj, double yi, double L) {
    double a = fabs(yj - yi);
    if (L - a < a) a = L - a;
    return a;
}

/* Time of flight of i (moving +x) towards j; INFINITY outside the corridor. */
static double time_of_flight(double xi, double yi, double xj, double yj,
                             double L, double d) {
    double a = perp_dist(yj, yi, L);
    if (!(a < d)) return INFINITY;
    double b = sqrt(d * d - a * a);
    double tau = fwd_dx(xj, xi, L) - b;
    if (tau < 0.0) tau = 0.0;
    return tau;
}

static double wrap_add(double x, double dx, double L) {
    double r = x + dx;
    if (r >= L) r -= L;
    return r;
}

/*
 * Corridor of j as seen from i (Sec. 3.1): 0 for |dy| < d/2, 1 for
 * d/2 <= dy < d, 2 for -d < dy <= -d/2, -1 for |dy| >= d; dy is the minimum
 * image of y_j - y_i, and |dy| is computed exactly as in perp_dist.
 */
static int corridor(double yj, double yi, double L, double d) {
    double dy = yj - yi;
    double a = fabs(dy);
    int flip = 0;
    if (L - a < a) {
        a = L - a;
        flip = 1;
    }
    if (!(a < d)) return -1;
    if (a < 0.5 * d) return 0;
    int up = dy > 0.0;
    if (flip) up = !up;
    return up ? 1 : 2;
}

/* End of claim window w of W in a leg of length ell (the last one is open). */
static double window_end(const orc_params *p, int w) {
    if (w + 1 >= p->windows) return INFINITY;
    return ((double)(w + 1) * p->ell) / (double)p->windows;
}

/* ---------------------------------------------------------------- cell lists */

typedef struct {
    int nc;
    double a, inv_a, eps;
    int32_t *head; /* [nc*nc], -1 = empty */
    int32_t *next; /* [n] */
} cells_t;

static int cell_coord(double v, const cells_t *g) {
    int c = (int)(v * g->inv_a);
    if (c >= g->nc) c = g->nc - 1;
    if (c < 0) c = 0;
    return c;
}

static int cell_of(double x, double y, const cells_t *g) {
    return cell_coord(y, g) * g->nc + cell_coord(x, g);
}

static void cell_insert(cells_t *g, int cell, int j) {
    g->next[j] = g->head[cell];
    g->head[cell] = j;
}

static void cell_remove(cells_t *g, int cell, int j) {
    int32_t *p = &g->head[cell];
    while (*p != j) p = &g->next[*p];
    *p = g->next[j];
}

static int cells_init(cells_t *g, const orc_params *p, const double *x,
                      const double *y) {
    g->nc = p->nc;
    g->a = p->L / (double)p->nc;
    g->inv_a = (double)p->nc / p->L;
    g->eps = ldexp(p->L, -30);
    size_t ncell = (size_t)p->nc * (size_t)p->nc;
    g->head = (int32_t *)malloc(ncell * sizeof(int32_t));
    g->next = (int32_t *)malloc((size_t)p->n * sizeof(int32_t));
    if (!g->head || !g->next) return -1;
    for (size_t q = 0; q < ncell; ++q) g->head[q] = -1;
    for (int64_t j = p->n - 1; j >= 0; --j)
        cell_insert(g, cell_of(x[j], y[j], g), (int)j);
    return 0;
}

static void cells_free(cells_t *g) {
    free(g->head);
    free(g->next);
}

/* Move disk j from its cell at (x_old, y) to the cell of (x_new, y). */
static void cell_move(cells_t *g, int j, double x_old, double x_new, double y) {
    int c0 = cell_of(x_old, y, g), c1 = cell_of(x_new, y, g);
    if (c0 != c1) {
        cell_remove(g, c0, j);
        cell_insert(g, c1, j);
    }
}

/* --------------------------------------------------------- one chain's step */

typedef struct {
    int lift;     /* 1: lift to j, 0: stall */
    int j;        /* target (lift only) */
    double tau;   /* tau* (lift) or D (stall) */
    int cx, cy;   /* scanned footprint: rows cy-1..cy+1, columns cx..cx+mlast */
    int mlast;
} step_t;

/* Candidate filter: exclude i itself; with tags, exclude non-static disks. */
static int is_candidate(int j, int i, const int8_t *tag) {
    if (j == i) return 0;
    if (tag && tag[j] != TAG_STATIC) return 0;
    return 1;
}

/* Lexicographic (tau, j) comparison for the argmin. */
static int better(double tau, int j, double btau, int bj) {
    return tau < btau || (tau == btau && j < bj);
}

/* All-pairs definition: argmin over every candidate disk. */
/* Time of flight in the lazily advanced frame of i: each chain's disk keeps
   (x_i, t_i) and moves only when its chain acts. A disk j with
   t_i + tau < t_j became static after i had passed its position (the horizon
   condition of Eq. 2 fails), so it is one lap away: tau + L. */
static double lazy_tof(const orc_params *p, const double *x, const double *y,
                       const double *t, int i, int j) {
    double tau = time_of_flight(x[i], y[i], x[j], y[j], p->L, p->d);
    if (tau != INFINITY && t[i] + tau < t[j]) tau = tau + p->L;
    return tau;
}

static step_t step_allpairs(const orc_params *p, const double *x, const double *y,
                            const double *t, const int8_t *tag, int i, double D) {
    double btau = INFINITY;
    int bj = INT32_MAX;
    for (int64_t j = 0; j < p->n; ++j) {
        if (!is_candidate((int)j, i, tag)) continue;
        double tau = lazy_tof(p, x, y, t, i, (int)j);
        if (tau == INFINITY) continue;
        if (better(tau, (int)j, btau, bj)) {
            btau = tau;
            bj = (int)j;
        }
    }
    step_t s;
    memset(&s, 0, sizeof s);
    if (btau < D) {
        s.lift = 1;
        s.j = bj;
        s.tau = btau;
    } else {
        s.lift = 0;
        s.j = -1;
        s.tau = D;
    }
    s.mlast = -1;
    return s;
}

/* Cell scan with the stop rule; claim(cell, ctx) is called for every scanned cell. */
typedef void (*claim_fn)(int cell, void *ctx);

static step_t step_cells(const orc_params *p, const cells_t *g, const double *x,
                         const double *y, const double *t, const int8_t *tag, int i,
                         double D, claim_fn claim, void *claim_ctx) {
    int nc = g->nc;
    int cx = cell_coord(x[i], g), cy = cell_coord(y[i], g);
    double fx = x[i] - (double)cx * g->a;
    int rows[3] = {(cy + nc - 1) % nc, cy, (cy + 1) % nc};
    double btau = INFINITY;
    int bj = INT32_MAX;
    int mlast = 0;
    for (int m = 0; m < nc; ++m) {
        if (m >= 1) {
            double best = btau < D ? btau : D;
            double thr = ((double)m * g->a - fx) - p->d;
            if (thr > best + g->eps) break;
        }
        int col = (cx + m) % nc;
        for (int r = 0; r < 3; ++r) {
            int cell = rows[r] * nc + col;
            if (claim) claim(cell, claim_ctx);
            for (int j = g->head[cell]; j >= 0; j = g->next[j]) {
                if (!is_candidate(j, i, tag)) continue;
                double tau = lazy_tof(p, x, y, t, i, j);
                if (tau == INFINITY) continue;
                if (better(tau, j, btau, bj)) {
                    btau = tau;
                    bj = j;
                }
            }
        }
        mlast = m;
    }
    step_t s;
    s.cx = cx;
    s.cy = cy;
    s.mlast = mlast;
    if (btau < D) {
        s.lift = 1;
        s.j = bj;
        s.tau = btau;
    } else {
        s.lift = 0;
        s.j = -1;
        s.tau = D;
    }
    return s;
}

static int in_footprint(const step_t *s, int cell, int nc) {
    int r = cell / nc, col = cell % nc;
    int dr = (r - s->cy + nc) % nc;
    if (!(dr == 0 || dr == 1 || dr == nc - 1)) return 0;
    int dm = (col - s->cx + nc) % nc;
    return dm <= s->mlast;
}

/* ------------------------------------------- constraint graph G(3), Sec. 3.1 */

/* Arrows of i by the definition: every other disk is examined. */
static void arrows_allpairs(const orc_params *p, const double *x, const double *y, int i,
                            int32_t out[3]) {
    double bt[3] = {INFINITY, INFINITY, INFINITY};
    int bj[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
    for (int64_t j = 0; j < p->n; ++j) {
        if (j == i) continue;
        int kc = corridor(y[j], y[i], p->L, p->d);
        if (kc < 0) continue;
        double tau = time_of_flight(x[i], y[i], x[j], y[j], p->L, p->d);
        if (better(tau, (int)j, bt[kc], bj[kc])) {
            bt[kc] = tau;
            bj[kc] = (int)j;
        }
    }
    for (int kc = 0; kc < 3; ++kc) out[kc] = bt[kc] == INFINITY ? -1 : bj[kc];
}

/*
 * Arrows of i by the cell scan: columns cx, cx+1, ... of rows cy-1..cy+1
 * (|dy| < d keeps j within one row of cells), stopping before column m >= 1
 * once (m*a - fx) - d exceeds the best tau of every corridor by eps (no disk
 * of a later column can then do better); a corridor that is still empty
 * makes the scan go once round the box.
 */
static void arrows_cells(const orc_params *p, const cells_t *g, const double *x,
                         const double *y, int i, int32_t out[3]) {
    int nc = g->nc;
    int cx = cell_coord(x[i], g), cy = cell_coord(y[i], g);
    double fx = x[i] - (double)cx * g->a;
    int rows[3] = {(cy + nc - 1) % nc, cy, (cy + 1) % nc};
    double bt[3] = {INFINITY, INFINITY, INFINITY};
    int bj[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
    for (int m = 0; m < nc; ++m) {
        if (m >= 1) {
            double worst = bt[0];
            if (bt[1] > worst) worst = bt[1];
            if (bt[2] > worst) worst = bt[2];
            double thr = ((double)m * g->a - fx) - p->d;
            if (thr > worst + g->eps) break;
        }
        int col = (cx + m) % nc;
        for (int r = 0; r < 3; ++r) {
            for (int j = g->head[rows[r] * nc + col]; j >= 0; j = g->next[j]) {
                if (j == i) continue;
                int kc = corridor(y[j], y[i], p->L, p->d);
                if (kc < 0) continue;
                double tau = time_of_flight(x[i], y[i], x[j], y[j], p->L, p->d);
                if (better(tau, j, bt[kc], bj[kc])) {
                    bt[kc] = tau;
                    bj[kc] = j;
                }
            }
        }
    }
    for (int kc = 0; kc < 3; ++kc) out[kc] = bt[kc] == INFINITY ? -1 : bj[kc];
}

/*
 * The graph as a step needs it: arrows of disk i from the configuration at
 * the start of the leg (x0 and its cells g0), computed on first use.
 */
typedef struct {
    const double *x0;
    const cells_t *g0;
    int32_t *arrow; /* [3n]; -2 = not computed yet */
} graph_t;

static const int32_t *graph_arrows(const orc_params *p, graph_t *G, const double *y, int i) {
    int32_t *a = G->arrow + 3 * (int64_t)i;
    if (a[0] == -2) arrows_cells(p, G->g0, G->x0, y, i, a);
    return a;
}

/*
 * The next event of the chain whose active disk is i (time of flight to each
 * candidate, Sec. 2.2, and the least (tau, j)), with the candidates taken
 * from the arrows of i; every disk read (i and each arrow target) is passed
 * to claim().
 */
static step_t step_graph(const orc_params *p, graph_t *G, const double *x, const double *y,
                         const double *t, const int8_t *tag, int i, double D,
                         claim_fn claim, void *claim_ctx) {
    const int32_t *a = graph_arrows(p, G, y, i);
    if (claim) claim(i, claim_ctx);
    double btau = INFINITY;
    int bj = INT32_MAX;
    for (int kc = 0; kc < 3; ++kc) {
        int j = a[kc];
        if (j < 0) continue;
        if (claim) claim(j, claim_ctx);
        if (!is_candidate(j, i, tag)) continue;
        double tau = lazy_tof(p, x, y, t, i, j);
        if (tau == INFINITY) continue;
        if (better(tau, j, btau, bj)) {
            btau = tau;
            bj = j;
        }
    }
    step_t s;
    memset(&s, 0, sizeof s);
    s.mlast = -1;
    if (btau < D) {
        s.lift = 1;
        s.j = bj;
        s.tau = btau;
    } else {
        s.lift = 0;
        s.j = -1;
        s.tau = D;
    }
    return s;
}

/* ------------------------------------------------ isolated runs (the flag) */

typedef struct {
    int32_t *owner; /* [ncell], first chain that scanned the cell, -1 none */
    int c;
    int conflict;
} claim_ctx_t;

static void claim_record(int cell, void *vctx) {
    claim_ctx_t *cc = (claim_ctx_t *)vctx;
    int32_t o = cc->owner[cell];
    if (o < 0)
        cc->owner[cell] = cc->c;
    else if (o != cc->c)
        cc->conflict = 1;
}

/*
 * Runs one chain alone from the current state -- its disk i0 at local time
 * t[i0], remaining length D; every other disk counts as static -- through its
 * events before t_end, recording the cells it scans (the last scan, whose
 * event lies at or after t_end, included); then restores x, t and the cells.
 */
static int64_t isolated_chain(const orc_params *p, cells_t *g, graph_t *G, double *x,
                              const double *y, double *t, int i0, double D0,
                              double t_end, claim_ctx_t *cc, int32_t *undo_i,
                              double *undo_x, double *undo_t, int64_t undo_cap,
                              int *overflow) {
    int i = i0;
    double D = D0;
    int64_t nu = 0, lifts = 0;
    for (;;) {
        step_t s = p->search == 2
                       ? step_graph(p, G, x, y, t, NULL, i, D, claim_record, cc)
                       : step_cells(p, g, x, y, t, NULL, i, D, claim_record, cc);
        if (!(t[i] + s.tau < t_end)) break;
        if (nu + 2 > undo_cap) {
            *overflow = 1;
            break;
        }
        undo_i[nu] = i;
        undo_x[nu] = x[i];
        undo_t[nu] = t[i];
        ++nu;
        if (s.lift) {
            undo_i[nu] = s.j;
            undo_x[nu] = x[s.j];
            undo_t[nu] = t[s.j];
            ++nu;
        }
        double tn = t[i] + s.tau;
        double xn = wrap_add(x[i], s.tau, p->L);
        cell_move(g, i, x[i], xn, y[i]);
        x[i] = xn;
        if (!s.lift) {
            t[i] = tn;
            break;
        }
        t[s.j] = tn;
        t[i] = tn;
        D = D - s.tau;
        i = s.j;
        ++lifts;
    }
    for (int64_t u = nu - 1; u >= 0; --u) {
        int j = undo_i[u];
        cell_move(g, j, x[j], undo_x[u], y[j]);
        x[j] = undo_x[u];
        t[j] = undo_t[u];
    }
    return lifts;
}

/* ------------------------------------------------------------ Alg. 2 (leg) */

typedef struct {
    double T; /* global event time */
    step_t s;
} event_t;

static void compute_event(const orc_params *p, const cells_t *g, graph_t *G,
                          const double *x, const double *y, const double *t,
                          const int8_t *tag, int i, double D, event_t *ev) {
    if (p->search == 0)
        ev->s = step_allpairs(p, x, y, t, tag, i, D);
    else if (p->search == 2)
        ev->s = step_graph(p, G, x, y, t, tag, i, D, NULL, NULL);
    else
        ev->s = step_cells(p, g, x, y, t, tag, i, D, NULL, NULL);
    ev->T = t[i] + ev->s.tau;
}

/*
 * One leg of Alg. 2 from leg-relative time 0 to ell.
 *   x      [n] in/out (positions along v); y [n] in (never changes for v=(1,0))
 *   t      [n] out: local times at the end of the leg (leg-relative)
 *   active [k] in/out: chain c's active disk
 *   log    optional lifting log (appended at *log_n, capacity log_cap)
 *   flag   out: 1 iff the isolated claim sets of two chains share a cell
 *          (search 0 or 1) or a disk (search 2), computed window by window
 *   lifts  out: number of liftings in this leg
 *   lifts_per_chain  optional [k] out: liftings of each chain
 *   wflags optional [windows] out: the flag of each claim window
 * Returns 0, or -1 on allocation failure, -2 on log/undo overflow,
 * -3 on bad parameters, -6 if an event was found earlier than the last one
 * executed (a broken global-time order; never expected).
 */
int orc_leg(const orc_params *p, int32_t leg, double *x, const double *y,
            double *t, int32_t k, int32_t *active, orc_lift *log,
            int64_t log_cap, int64_t *log_n, uint8_t *flag, int64_t *lifts,
            int64_t *lifts_per_chain, uint8_t *wflags) {
    if (p->n <= 0 || k <= 0 || k > p->n || p->nc < 3) return -3;
    if (!(p->L / (double)p->nc > p->d)) return -3;
    int64_t n = p->n;
    int nc = p->nc;
    cells_t g;
    if (cells_init(&g, p, x, y)) return -1;
    int8_t *tag = (int8_t *)calloc((size_t)n, 1);
    double *D = (double *)malloc((size_t)k * sizeof(double));
    int8_t *run = (int8_t *)malloc((size_t)k);
    event_t *ev = (event_t *)malloc((size_t)k * sizeof(event_t));
    /* claim owners: per cell, or per disk with the constraint graph */
    int64_t n_claim = p->search == 2 ? n : (int64_t)nc * nc;
    int32_t *owner = (int32_t *)malloc((size_t)n_claim * sizeof(int32_t));
    /* constraint graph: arrows from the leg-start configuration */
    graph_t G = {NULL, NULL, NULL};
    double *x0 = NULL;
    cells_t g0;
    int have_g0 = 0;
    int64_t undo_cap = 1 << 20;
    int32_t *undo_i = (int32_t *)malloc((size_t)undo_cap * sizeof(int32_t));
    double *undo_x = (double *)malloc((size_t)undo_cap * sizeof(double));
    double *undo_t = (double *)malloc((size_t)undo_cap * sizeof(double));
    int rc = 0;
    if (!tag || !D || !run || !ev || !owner || !undo_i || !undo_x || !undo_t) {
        rc = -1;
        goto done;
    }

    if (p->windows < 1) {
        rc = -3;
        goto done;
    }
    if (p->search == 2) {
        x0 = (double *)malloc((size_t)n * sizeof(double));
        G.arrow = (int32_t *)malloc((size_t)n * 3 * sizeof(int32_t));
        if (!x0 || !G.arrow || cells_init(&g0, p, x, y)) {
            rc = -1;
            goto done;
        }
        have_g0 = 1;
        memcpy(x0, x, (size_t)n * sizeof(double));
        for (int64_t q = 0; q < 3 * n; ++q) G.arrow[q] = -2;
        G.x0 = x0;
        G.g0 = &g0;
    }
    for (int64_t j = 0; j < n; ++j) t[j] = 0.0;
    for (int c = 0; c < k; ++c) {
        tag[active[c]] = TAG_ACTIVE;
        D[c] = p->ell;
        run[c] = 1;
        if (lifts_per_chain) lifts_per_chain[c] = 0;
    }
    for (int c = 0; c < k; ++c)
        compute_event(p, &g, &G, x, y, t, tag, active[c], D[c], &ev[c]);
    int64_t nl = 0;
    double now = 0.0;
    int any_conflict = 0;
    for (int w = 0; w < p->windows; ++w) {
        const double t_end = window_end(p, w);
        /* conflict flag of the window: isolated runs from the current state */
        {
            for (int64_t q = 0; q < n_claim; ++q) owner[q] = -1;
            claim_ctx_t cc;
            cc.owner = owner;
            cc.conflict = 0;
            int overflow = 0;
            for (int c = 0; c < k; ++c) {
                if (!run[c]) continue;
                cc.c = c;
                isolated_chain(p, &g, &G, x, y, t, active[c], D[c], t_end, &cc, undo_i,
                               undo_x, undo_t, undo_cap, &overflow);
            }
            if (overflow) {
                rc = -2;
                goto done;
            }
            any_conflict |= cc.conflict;
            if (wflags) wflags[w] = (uint8_t)cc.conflict;
        }
        /* Alg. 2: the events of the window in global-time order */
        for (;;) {
            int cb = -1;
            for (int c = 0; c < k; ++c) {
                if (!run[c]) continue;
                if (cb < 0 || ev[c].T < ev[cb].T) cb = c;
            }
            if (cb < 0 || !(ev[cb].T < t_end)) break;
            /* events come in global-time order: nothing recomputed lies in the past */
            if (ev[cb].T < now) {
                rc = -6;
                goto done;
            }
            now = ev[cb].T;
            int i = active[cb];
            step_t s = ev[cb].s;
            double x_old = x[i];
            int changed[3];
            int nchanged = 0;
            changed[nchanged++] = cell_of(x_old, y[i], &g);
            if (s.lift) {
                /* lifting i -> j (Eq. 1): i moves by tau to contact with j,
                   both now carry the event's local time, activity passes to
                   j and the chain has tau less to go. The local times are
                   set before x moves (Remark 11). */
                int j = s.j;
                double tnew = t[i] + s.tau;
                t[j] = tnew;
                t[i] = tnew;
                double xn = wrap_add(x[i], s.tau, p->L);
                cell_move(&g, i, x[i], xn, y[i]);
                x[i] = xn;
                tag[i] = TAG_STATIC;
                D[cb] = D[cb] - s.tau;
                tag[j] = TAG_ACTIVE;
                active[cb] = j;
                changed[nchanged++] = cell_of(xn, y[i], &g);
                changed[nchanged++] = cell_of(x[j], y[j], &g);
                if (log) {
                    if (*log_n >= log_cap) {
                        rc = -2;
                        goto done;
                    }
                    orc_lift *e = &log[(*log_n)++];
                    e->leg = leg;
                    e->c = cb;
                    e->i = i;
                    e->j = j;
                    e->t = tnew;
                    e->tau = s.tau;
                    e->xi = xn;
                    e->xj = x[j];
                }
                ++nl;
                if (lifts_per_chain) lifts_per_chain[cb] += 1;
            } else {
                /* no contact within the remaining length D: i moves by D and
                   stalls with local time h' (Remark 1); it starts the
                   chain's next leg */
                t[i] = t[i] + D[cb];
                double xn = wrap_add(x[i], D[cb], p->L);
                cell_move(&g, i, x[i], xn, y[i]);
                x[i] = xn;
                D[cb] = 0.0;
                tag[i] = TAG_STALLED;
                run[cb] = 0;
                changed[nchanged++] = cell_of(xn, y[i], &g);
            }
            /* recompute the events that the change can affect (all of them
               without a cell footprint to test against) */
            for (int c = 0; c < k; ++c) {
                if (!run[c]) continue;
                int redo = (c == cb) || p->search != 1;
                for (int q = 0; q < nchanged && !redo; ++q)
                    if (in_footprint(&ev[c].s, changed[q], nc)) redo = 1;
                if (redo) compute_event(p, &g, &G, x, y, t, tag, active[c], D[c], &ev[c]);
            }
        }
    }
    if (flag) *flag = (uint8_t)any_conflict;
    if (lifts) *lifts = nl;
done:
    cells_free(&g);
    if (have_g0) cells_free(&g0);
    free(x0);
    free(G.arrow);
    free(tag);
    free(D);
    free(run);
    free(ev);
    free(owner);
    free(undo_i);
    free(undo_x);
    free(undo_t);
    return rc;
}

/* --------------------------------------------------------------- Alg. 4 */

/*
 * Alg. 4 (single-threaded, local times) over one leg, all-pairs candidates.
 * The lowest-index chain whose disk has not reached ell, and that is not
 * waiting behind an active disk, runs until it stalls or would lift onto an
 * active disk (then it moves up to contact and waits, Remark 10). Waiting
 * chains are retried after any other chain has moved.
 * Returns 0 on success, 1 if a horizon violation aborted the run,
 * -1 on allocation failure, -2 on log overflow, -4 if every unfinished chain
 * waits behind an active disk (a necklace).
 */
int orc_alg4_leg(const orc_params *p, int32_t leg, double *x, const double *y,
                 double *t, int32_t k, int32_t *active, orc_lift *log,
                 int64_t log_cap, int64_t *log_n) {
    int64_t n = p->n;
    int8_t *tag = (int8_t *)calloc((size_t)n, 1);
    double *D = (double *)malloc((size_t)k * sizeof(double));
    int8_t *waiting = (int8_t *)calloc((size_t)k, 1);
    int rc = 0;
    if (!tag || !D || !waiting) {
        rc = -1;
        goto done;
    }
    for (int64_t j = 0; j < n; ++j) t[j] = 0.0;
    for (int c = 0; c < k; ++c) {
        tag[active[c]] = TAG_ACTIVE;
        D[c] = p->ell;
    }
    for (;;) {
        int c = -1, unfinished = 0;
        for (int q = 0; q < k; ++q) {
            if (!(D[q] > 0.0)) continue;
            unfinished = 1;
            if (!waiting[q]) {
                c = q;
                break;
            }
        }
        if (!unfinished) break;
        if (c < 0) {
            rc = -4;
            goto done;
        }
        int moved = 0;
        for (;;) {
            int i = active[c];
            double btau = INFINITY;
            int bj = INT32_MAX;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double tau = time_of_flight(x[i], y[i], x[j], y[j], p->L, p->d);
                if (tau == INFINITY) continue;
                if (t[i] + tau < t[j]) { /* horizon condition violated */
                    rc = 1;
                    goto done;
                }
                if (better(tau, (int)j, btau, bj)) {
                    btau = tau;
                    bj = (int)j;
                }
            }
            if (!(btau < D[c])) { /* stall at ell */
                t[i] = t[i] + D[c];
                x[i] = wrap_add(x[i], D[c], p->L);
                D[c] = 0.0;
                tag[i] = TAG_STALLED;
                moved = 1;
                break;
            }
            if (tag[bj] != TAG_STATIC) { /* target active: up to contact, wait */
                if (btau > 0.0) moved = 1;
                t[i] = t[i] + btau;
                x[i] = wrap_add(x[i], btau, p->L);
                D[c] = D[c] - btau;
                waiting[c] = 1;
                break;
            }
            double tnew = t[i] + btau;
            t[bj] = tnew;
            t[i] = tnew;
            x[i] = wrap_add(x[i], btau, p->L);
            tag[i] = TAG_STATIC;
            D[c] = D[c] - btau;
            tag[bj] = TAG_ACTIVE;
            active[c] = bj;
            moved = 1;
            if (log) {
                if (*log_n >= log_cap) {
                    rc = -2;
                    goto done;
                }
                orc_lift *e = &log[(*log_n)++];
                e->leg = leg;
                e->c = c;
                e->i = i;
                e->j = bj;
                e->t = tnew;
                e->tau = btau;
                e->xi = x[i];
                e->xj = x[bj];
            }
        }
        if (moved)
            for (int q = 0; q < k; ++q)
                if (q != c) waiting[q] = 0;
    }
done:
    free(tag);
    free(D);
    free(waiting);
    return rc;
}

/* ------------------------------------------------------ exported helpers */

/* Step function alone (for tests): argmin over all pairs and over cells. */
int orc_step(const orc_params *p, const double *x, const double *y,
             const double *t_or_null, const int8_t *tag, int32_t i, double D,
             int32_t *lift, int32_t *j, double *tau, int32_t *mlast) {
    step_t s;
    double *tz = NULL;
    const double *t = t_or_null;
    if (!t) {
        tz = (double *)calloc((size_t)p->n, sizeof(double));
        if (!tz) return -1;
        t = tz;
    }
    if (p->search == 0) {
        s = step_allpairs(p, x, y, t, tag, i, D);
    } else {
        cells_t g;
        if (cells_init(&g, p, x, y)) {
            free(tz);
            return -1;
        }
        s = step_cells(p, &g, x, y, t, tag, i, D, NULL, NULL);
        cells_free(&g);
    }
    free(tz);
    *lift = s.lift;
    *j = s.j;
    *tau = s.tau;
    *mlast = s.mlast;
    return 0;
}

/* The cells one isolated chain scans (claim set), for tests of the flag. */
typedef struct {
    int32_t *cells;
    int64_t cap, n;
    int32_t *seen;
} collect_ctx_t;

static void claim_collect(int cell, void *vctx) {
    collect_ctx_t *cc = (collect_ctx_t *)vctx;
    if (cc->seen[cell]) return;
    cc->seen[cell] = 1;
    if (cc->n < cc->cap) cc->cells[cc->n] = cell;
    cc->n++;
}

int orc_claim_set(const orc_params *p, const double *x_in, const double *y,
                  int32_t i0, int32_t *cells, int64_t cap, int64_t *n_out) {
    int64_t n = p->n;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    int32_t *seen = (int32_t *)calloc((size_t)p->nc * p->nc, sizeof(int32_t));
    if (!x || !seen) {
        free(x);
        free(seen);
        return -1;
    }
    memcpy(x, x_in, (size_t)n * sizeof(double));
    cells_t g;
    if (cells_init(&g, p, x, y)) {
        free(x);
        free(seen);
        return -1;
    }
    double *t = (double *)calloc((size_t)n, sizeof(double));
    if (!t) {
        cells_free(&g);
        free(x);
        free(seen);
        return -1;
    }
    collect_ctx_t cc = {cells, cap, 0, seen};
    int i = i0;
    double D = p->ell;
    for (;;) {
        step_t s = step_cells(p, &g, x, y, t, NULL, i, D, claim_collect, &cc);
        double xn = wrap_add(x[i], s.tau, p->L);
        cell_move(&g, i, x[i], xn, y[i]);
        x[i] = xn;
        if (!s.lift) break;
        t[s.j] = t[i] + s.tau;
        t[i] = t[i] + s.tau;
        D = D - s.tau;
        i = s.j;
    }
    *n_out = cc.n;
    cells_free(&g);
    free(x);
    free(t);
    free(seen);
    return cc.n > cap ? -2 : 0;
}

/*
 * Arrows of the constraint graph G(3) (Sec. 3.1) for the disks ids[0..m-1]
 * (for every disk when ids is NULL; m is then ignored): out[3q + kc] is the
 * target in corridor kc (0 centre, 1 upper, 2 lower) or -1 when the corridor
 * is empty. search 0: by the definition, every pair; search 1: by the cell
 * scan that orc_leg uses with search == 2.
 */
int orc_graph3(const orc_params *p, const double *x, const double *y, int32_t search,
               const int32_t *ids, int64_t m, int32_t *out) {
    if (p->n <= 0 || p->nc < 3 || !(p->L / (double)p->nc > p->d)) return -3;
    const int64_t cnt = ids ? m : p->n;
    cells_t g;
    int have = 0;
    if (search != 0) {
        if (cells_init(&g, p, x, y)) return -1;
        have = 1;
    }
    for (int64_t q = 0; q < cnt; ++q) {
        const int i = ids ? ids[q] : (int)q;
        if (i < 0 || i >= p->n) {
            if (have) cells_free(&g);
            return -3;
        }
        if (search == 0)
            arrows_allpairs(p, x, y, i, out + 3 * q);
        else
            arrows_cells(p, &g, x, y, i, out + 3 * q);
    }
    if (have) cells_free(&g);
    return 0;
}
