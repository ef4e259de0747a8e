/*
 * alg5_openmp.c -- CPU baseline: the paper's multithreaded ECMC with local
 * times (Alg. 5, Sec. 3) restated for the host cores with OpenMP threads.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE, not an oracle: with several chains in
 * flight its output depends on the thread schedule. It is timed by the
 * benchmark as the multicore CPU baseline (the paper's own design on the
 * box's host cores); the tests pin its single-thread, single-chain runs to
 * the oracle (Alg. 2 and Alg. 4 coincide then). It shares no code with the
 * CUDA path.
 *
 * What one leg does (Alg. 5, one task per chain, tasks spread over threads):
 *   - every disk's local time is reset to 0 and the start disk of each chain
 *     is tagged active (the lifted configuration at the breakpoint);
 *   - a chain repeats: scan the cells ahead of its active disk i (rows
 *     cy-1..cy+1, columns cx, cx+1, ... with the same stop rule as the
 *     oracle), time of flight tau_j = dx - sqrt(d^2 - dy^2) for static disks
 *     in the corridor (Sec. 2.2), horizon check t_i + tau_j < t_j (Eq. 2:
 *     counted as a violation; the disk is then taken one lap away as in the
 *     oracle's lazy frame), argmin of (tau, j);
 *     lift if tau* < D: compare-and-swap of j's tag from static to active
 *     (a failed swap is a violation and the chain scans again), then t_j,
 *     t_i, x_i, D and i <- j (the lifting of Eq. 1, local times before the
 *     position as Remark 11 requires); otherwise move by D and stall;
 *   - tags are acquire/release (the paper's validation ordering, Sec. 4);
 *     positions and local times are relaxed atomics, cells are fixed-size
 *     slot arrays updated with compare-and-swap.
 * A violation does not stop the leg (the paper's benchmark mode): the count
 * is returned with the liftings.
 *
 * Compile: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define A5_STATIC 0
#define A5_SLOTS 8

typedef struct {
    int64_t n;
    double L, d, ell;
    int32_t nc;      /* cells per side (cell side L/nc > d) */
    int32_t threads; /* 0 = all */
} a5_params;

typedef struct {
    int32_t nc;
    double inv_a, a;
    int32_t *slot; /* [nc*nc*A5_SLOTS], -1 = empty */
} a5_cells;

static double ld(const double *p) {
    double v;
    __atomic_load(p, &v, __ATOMIC_RELAXED);
    return v;
}

static void st(double *p, double v) { __atomic_store(p, &v, __ATOMIC_RELAXED); }

static int coord(double v, const a5_cells *g) {
    int c = (int)(v * g->inv_a);
    if (c >= g->nc) c = g->nc - 1;
    if (c < 0) c = 0;
    return c;
}

static int cell_of(double x, double y, const a5_cells *g) {
    return coord(y, g) * g->nc + coord(x, g);
}

static int slot_insert(a5_cells *g, int cell, int32_t j) {
    int32_t *s = g->slot + (int64_t)cell * A5_SLOTS;
    for (int q = 0; q < A5_SLOTS; ++q) {
        int32_t e = -1;
        if (__atomic_compare_exchange_n(s + q, &e, j, 0, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED))
            return 0;
    }
    return -1;
}

static void slot_remove(a5_cells *g, int cell, int32_t j) {
    int32_t *s = g->slot + (int64_t)cell * A5_SLOTS;
    for (int q = 0; q < A5_SLOTS; ++q) {
        int32_t e = j;
        if (__atomic_compare_exchange_n(s + q, &e, -1, 0, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED))
            return;
    }
}

/* One chain from its start disk through the leg (Alg. 5, one task). */
static void run_chain(const a5_params *p, a5_cells *g, double *x, const double *y, double *t,
                      int32_t *tag, int32_t c, int32_t *active, int64_t *lifts,
                      int64_t *violations) {
    const int nc = g->nc;
    const double eps = p->L * 0x1p-30;
    int32_t i = active[c];
    double D = p->ell;
    double ti = 0.0;
    int64_t nl = 0, nv = 0;
    for (;;) {
        const double xi = ld(x + i), yi = y[i];
        const int cx = coord(xi, g), cy = coord(yi, g);
        const double fx = xi - (double)cx * g->a;
        const int rows[3] = {(cy + nc - 1) % nc, cy, (cy + 1) % nc};
        double btau = INFINITY;
        int32_t bj = INT32_MAX;
        for (int m = 0; m < nc; ++m) {
            if (m >= 1) {
                const double best = btau < D ? btau : D;
                if (((double)m * g->a - fx) - p->d > best + eps) break;
            }
            const int col = (cx + m) % nc;
            for (int r = 0; r < 3; ++r) {
                const int32_t *s = g->slot + (int64_t)(rows[r] * nc + col) * A5_SLOTS;
                for (int q = 0; q < A5_SLOTS; ++q) {
                    const int32_t j = __atomic_load_n(s + q, __ATOMIC_RELAXED);
                    if (j < 0 || j == i) continue;
                    if (__atomic_load_n(tag + j, __ATOMIC_ACQUIRE) != A5_STATIC) continue;
                    double a = fabs(y[j] - yi);
                    if (p->L - a < a) a = p->L - a;
                    if (!(a < p->d)) continue;
                    const double b = sqrt(p->d * p->d - a * a);
                    double dx = ld(x + j) - xi;
                    if (dx < 0.0) dx += p->L;
                    double tau = dx - b;
                    if (tau < 0.0) tau = 0.0;
                    if (ti + tau < ld(t + j)) {  /* Eq. 2 fails: horizon violation */
                        ++nv;
                        tau = tau + p->L;
                    }
                    if (tau < btau || (tau == btau && j < bj)) {
                        btau = tau;
                        bj = j;
                    }
                }
            }
        }
        const int cell_i = cy * nc + cx;
        if (btau < D) {
            int32_t e = A5_STATIC;
            if (!__atomic_compare_exchange_n(tag + bj, &e, c + 1, 0, __ATOMIC_ACQ_REL,
                                             __ATOMIC_ACQUIRE)) {
                ++nv;  /* the target was taken by another chain: scan again */
                continue;
            }
            const double tnew = ti + btau;
            double xnew = xi + btau;
            if (xnew >= p->L) xnew -= p->L;
            st(t + bj, tnew);
            st(t + i, tnew);
            st(x + i, xnew);
            const int cell_new = cell_of(xnew, yi, g);
            if (cell_new != cell_i) {
                if (slot_insert(g, cell_new, i) != 0) ++nv; /* cell full: counted */
                slot_remove(g, cell_i, i);
            }
            __atomic_store_n(tag + i, A5_STATIC, __ATOMIC_RELEASE);
            D = D - btau;
            ti = tnew;
            i = bj;
            ++nl;
        } else {
            const double tnew = ti + D;
            double xnew = xi + D;
            if (xnew >= p->L) xnew -= p->L;
            st(t + i, tnew);
            st(x + i, xnew);
            const int cell_new = cell_of(xnew, yi, g);
            if (cell_new != cell_i) {
                if (slot_insert(g, cell_new, i) != 0) ++nv;
                slot_remove(g, cell_i, i);
            }
            break;  /* stalled: i stays tagged (active for the next leg) */
        }
    }
    active[c] = i;
    *lifts += nl;
    *violations += nv;
}

/*
 * n_legs legs of k chains from positions x (updated in place), y, start disks
 * active[k] (updated to the next legs' start disks). Returns 0, or -1 on bad
 * input / -2 on allocation failure / -3 when a cell overflows at the start.
 * *seconds is the wall time of the legs (monotonic clock), *threads_out the
 * threads used.
 */
int a5_run(const a5_params *p, double *x, const double *y, int32_t *active, int32_t k,
           int32_t n_legs, int64_t *lifts_out, int64_t *violations_out, double *seconds,
           int32_t *threads_out) {
    if (!p || p->n < 2 || p->nc < 3 || k < 1 || !(p->L / p->nc > p->d)) return -1;
    a5_cells g;
    g.nc = p->nc;
    g.a = p->L / (double)p->nc;
    g.inv_a = (double)p->nc / p->L;
    const int64_t ncell = (int64_t)p->nc * p->nc;
    g.slot = (int32_t *)malloc(sizeof(int32_t) * ncell * A5_SLOTS);
    double *t = (double *)calloc((size_t)p->n, sizeof(double));
    int32_t *tag = (int32_t *)calloc((size_t)p->n, sizeof(int32_t));
    if (!g.slot || !t || !tag) {
        free(g.slot);
        free(t);
        free(tag);
        return -2;
    }
    memset(g.slot, 0xff, sizeof(int32_t) * ncell * A5_SLOTS);
    for (int64_t j = 0; j < p->n; ++j)
        if (slot_insert(&g, cell_of(x[j], y[j], &g), (int32_t)j) != 0) {
            free(g.slot);
            free(t);
            free(tag);
            return -3;
        }
    int nth = 1;
#ifdef _OPENMP
    nth = p->threads > 0 ? p->threads : omp_get_max_threads();
#endif
    struct timespec c0, c1;
    clock_gettime(CLOCK_MONOTONIC, &c0);
    int64_t lifts = 0, viol = 0;
    for (int32_t leg = 0; leg < n_legs; ++leg) {
#pragma omp parallel for num_threads(nth) schedule(static)
        for (int64_t j = 0; j < p->n; ++j) {
            t[j] = 0.0;
            tag[j] = A5_STATIC;
        }
        for (int32_t c = 0; c < k; ++c) tag[active[c]] = c + 1;
#pragma omp parallel for num_threads(nth) schedule(dynamic, 1) reduction(+ : lifts, viol)
        for (int32_t c = 0; c < k; ++c) run_chain(p, &g, x, y, t, tag, c, active, &lifts, &viol);
    }
    clock_gettime(CLOCK_MONOTONIC, &c1);
    *seconds = (double)(c1.tv_sec - c0.tv_sec) + 1e-9 * (double)(c1.tv_nsec - c0.tv_nsec);
    *lifts_out = lifts;
    *violations_out = viol;
    *threads_out = nth;
    free(g.slot);
    free(t);
    free(tag);
    return 0;
}
