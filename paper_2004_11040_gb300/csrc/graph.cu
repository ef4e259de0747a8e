// graph.cu -- libecmc's constraint-graph path (ECMC_GRAPH): the liftings of
// a chain are found through the arrows of the constraint graph G(3) of
// Sec. 3.1 instead of a scan of the cells ahead.
//
// For v = (1, 0) the arrows of disk i are, in each of three corridors of
// dy = y_j - y_i (minimum image) -- centre |dy| < d/2, upper d/2 <= dy < d,
// lower -d < dy <= -d/2 -- the disk of least time of flight (tau, j), if any.
// Disks closer than d in y cannot pass one another while v holds, so the
// arrows stay valid across breakpoints (Sec. 3.1) and a step reads at most
// three target disks; b_ij = sqrt(d^2 - dy^2) is fixed with the arrow and
// stored beside it, so the step does no square root.
//
// Layout: one 64-byte record per disk (x, local time, owner word, three arrows
// and their b); y and the claim words in arrays of their own (y never
// changes along +x; the claims are cleared window by window).
//
// Conflicts are claims on disks instead of cells: within a claim window a
// chain claims (atomicCAS of the disk's claim word from 0 to chain + 1; the
// words are cleared between windows) every disk a step reads -- its active
// disk and the arrow targets -- and uses what it read only once the claims
// stand. A disk is therefore written only by its claimer
// during a window, a chain that meets another chain's claim stops, and
// without a meeting each chain follows the path it takes alone, which is the
// global-time result (Lemma 2). The leg's flag is 1 iff the disks that two
// chains read, each run alone from the window's start, overlap. Chains that
// met are rolled back to the earliest time one of them stopped and replayed
// in global event-time order (Alg. 2), one warp per conflict component, as on
// the cell path.
//
// All FP64 arithmetic uses explicit round-to-nearest intrinsics (the file is
// compiled with -fmad=false) so that results are reproducible bit for bit.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "devmem.h"
#include "graph.h"

namespace {

// chains are numbered by the owner word's 30 bits
constexpr int MAX_CHAINS = (int)OWN_CHAIN;

struct __align__(64) GDisk {
    double x, t;    // position along the motion; local time (leg-relative)
    uint32_t own;   // owner word (static / active / stalled + chain)
    uint32_t pad0;
    uint32_t a[3];  // arrows: centre, upper, lower corridor (NONE: empty)
    uint32_t pad1;
    double b[3];    // b_ij = sqrt(d^2 - dy^2) of each arrow
};
static_assert(sizeof(GDisk) == 64, "one disk record is one 64-byte line");

// One event of a chain: enough to undo it exactly, and the lifting (Eq. 1).
struct GEv {
    uint32_t i, j, seq, pad;  // moved disk, target (NONE: stall), application order
    double x_old;             // x of i before the move
    double ti_old, tj_old;    // local times of i and j before the event
    double t, tau, xi, xj;    // event time (= new t_j), time of flight, x_i at contact, x_j
    double d_after;           // remaining chain length after the event
};

struct GDev {
    int64_t n;
    int k, cap, windows, nc;
    double L, d, ell;
    GDisk *g;        // [n]
    double *y;       // [n]
    uint32_t *claim; // [n] 0, or chain + 1 holding the disk in this window
    // per chain
    uint32_t *ci, *ci0;  // active disk now / at the leg start
    double *D, *tc;
    int32_t *status, *partner, *nrec, *nlift;
    GEv *rec;  // [k * cap]
    // pending events of the replay, and the arrows they were computed from
    double *ev_T, *ev_tau, *ev_xj, *ev_tj;
    uint32_t *ev_j, *ev_a;  // ev_a: [3k]
    int32_t *ev_lift;
    // conflict components (names as the union-find of common.cuh expects)
    double *vt;
    int32_t *uf, *fin, *comp_of, *abort_to, *comp_cnt, *comp_off, *comp_root, *comp_mem, *ctl;
    int32_t *nabort;  // [2] components that met another chain, by round parity
    uint64_t *memb;   // (window, round) << 32 | root of the component listing the chain
    int restart;      // conflicts by restart strategy 2 (Sec. 3.4) instead of local repair
    double *tstar;    // [1] restart mode: the earliest stop time of a pass
    unsigned long long *lc;      // [LC_N]
    unsigned long long *tc_cnt;  // [TC_N]
    ecmc_lift_t *log;
    int64_t log_cap;
    int log_on;
    double *dbg;  // [16] first failed internal check
};
// Record e of chain c, stored by event index, then chain (the first events of
// a leg of all chains lie in one dense block).
__device__ __forceinline__ GEv *grec_at(const GDev &s, int c, int e) {
    return s.rec + (size_t)e * (size_t)s.k + (size_t)c;
}


__device__ void gdiag(const GDev &s, int kind, double a, double b, double c, double d,
                      double e, double f) {
    if (!s.dbg) return;
    if (atomicCAS((unsigned long long *)s.dbg, 0ull,
                  (unsigned long long)__double_as_longlong((double)kind)) != 0ull)
        return;
    s.dbg[1] = a;
    s.dbg[2] = b;
    s.dbg[3] = c;
    s.dbg[4] = d;
    s.dbg[5] = e;
    s.dbg[6] = f;
}

// Requests a disk record into this SM's L1 ahead of its load (no registers
// held; the load that follows may still go to L2).
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ double wrap_add(double x, double dx, double L) {
    double r = __dadd_rn(x, dx);
    if (dbits(r) >= dbits(L)) r = __dsub_rn(r, L);  // r >= 0
    return r;
}

// ------------------------------------------------------------ graph build

struct GBuild {
    int64_t n;
    int nc, nb;
    double L, d, d2, a, inv_a, eps, w;  // cells of side a; y bins of width w
    float Lf, wf, inv_wf, half_f, d_f;     // the same in FP32 (bins only)
    float dcut_f;        // d + a margin above the FP32 error of |dy| (slot filter)
    const double *x, *y;
    uint32_t *cid;       // [nc*nc*C] disk per slot, EMPTY
    double *cx, *cy;     // [nc*nc*C]
    float *cyf;          // [nc*nc*C] y in FP32
    int32_t *bins;       // [nb + 1]: counts, then their exclusive prefix
    GDisk *g;
    unsigned long long *err;  // cell overflow count
};

__device__ __forceinline__ int cell_coord(double v, double inv_a, int nc) {
    int c = __double2int_rz(__dmul_rn(v, inv_a));
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

template <int C>
__global__ void k_gb_cells(GBuild b) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= b.n) return;
    const double x = b.x[q], y = b.y[q];
    const uint32_t cell = (uint32_t)cell_coord(y, b.inv_a, b.nc) * (uint32_t)b.nc +
                          (uint32_t)cell_coord(x, b.inv_a, b.nc);
    // bins only need a monotone map of y, the same as in band_count: FP32
    int bin = __float2int_rz(__fmul_rn(__double2float_rn(y), b.inv_wf));
    if (bin >= b.nb) bin = b.nb - 1;
    if (bin < 0) bin = 0;
    atomicAdd(b.bins + bin, 1);
    for (int sl = 0; sl < C; ++sl) {
        const uint32_t loc = cell * C + sl;
        if (atomicCAS(b.cid + loc, EMPTY, (uint32_t)q) == EMPTY) {
            b.cx[loc] = x;
            b.cy[loc] = y;
            b.cyf[loc] = __double2float_rn(y);
            return;
        }
    }
    atomicAdd(b.err, 1ull);
}

// Exclusive prefix of the y-bin counts, in tiles of SCAN_TILE bins (one block
// of 1024 threads, 4 consecutive bins per thread): k_gb_tile_sums adds each
// tile, k_gb_scan_tiles scans each tile from the sum of the tiles before it;
// the last tile also writes the total to bins[nb].
constexpr int SCAN_TILE = 4096;

__device__ __forceinline__ int tile_bin(const GBuild &b, int64_t q) {
    return q < b.nb ? b.bins[q] : 0;
}

__global__ void k_gb_tile_sums(GBuild b, int32_t *part) {
    __shared__ int warp_tot[32];
    __shared__ int tot[2];
    const int64_t q0 = (int64_t)blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    const int v = tile_bin(b, q0) + tile_bin(b, q0 + 1) + tile_bin(b, q0 + 2) + tile_bin(b, q0 + 3);
    block_exscan(v, warp_tot, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
}

__global__ void k_gb_scan_tiles(GBuild b, const int32_t *part) {
    __shared__ int warp_tot[32];
    __shared__ int tot[2];
    __shared__ int base;
    if (threadIdx.x < 32) {  // sum of the tiles before this one
        int acc = 0;
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += 32) acc += part[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (threadIdx.x == 0) base = acc;
    }
    const int64_t q0 = (int64_t)blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    const int v0 = tile_bin(b, q0), v1 = tile_bin(b, q0 + 1), v2 = tile_bin(b, q0 + 2),
              v3 = tile_bin(b, q0 + 3);
    const int off = block_exscan(v0 + v1 + v2 + v3, warp_tot, tot) + base;
    const int o[4] = {off, off + v0, off + v0 + v1, off + v0 + v1 + v2};
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (q0 + u < b.nb) b.bins[q0 + u] = o[u];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) b.bins[b.nb] = base + tot[0];
}

// Disks whose y falls in a bin that meets [lo, hi) (periodic, hi - lo < L):
// an upper bound on the disks with y in that range. FP32 is enough: the map
// to bins is monotone, and the callers' one-bin margin (d/128) is far above
// the FP32 rounding of y, lo and hi.
__device__ int band_count(const GBuild &b, float lo, float hi) {
    if (lo < 0.f) {
        lo = __fadd_rn(lo, b.Lf);
        hi = __fadd_rn(hi, b.Lf);
    } else if (lo >= b.Lf) {
        lo = __fsub_rn(lo, b.Lf);
        hi = __fsub_rn(hi, b.Lf);
    }
    auto bin = [&](float v) {
        int q = __float2int_rz(__fmul_rn(v, b.inv_wf));
        return min(max(q, 0), b.nb - 1);
    };
    const int b0 = bin(lo);
    if (hi <= b.Lf) return b.bins[bin(hi) + 1] - b.bins[b0];
    return (b.bins[b.nb] - b.bins[b0]) + (b.bins[bin(__fsub_rn(hi, b.Lf)) + 1] - b.bins[0]);
}

// Arrows of G(3), one thread per disk: the thread scans the columns ahead
// (rows cy-1..cy+1) and keeps, per corridor, the least (tau, j). Before
// column m >= 1, if (m a - fx) - d exceeds the worst best tau of the
// corridors still in play (+ eps), no later column can improve any of them
// and the scan stops; a corridor that the y bins show empty is not in play,
// any other one keeps the scan going (once round the box at most).
// The FP64 pipe costs the same per warp instruction whatever the number of
// active lanes, so every lane takes a disk of its own, and two tests keep
// FP64 work off the slots that cannot matter, both exact:
// - |dy| in FP32 above d plus a margin larger than its rounding error: the
//   slot lies in no corridor;
// - RN(dx - d) above the corridor's best: the computed tau = RN(dx - b) with
//   b = RN(sqrt(d^2 - dy^2)) <= d is at least that (rounding is monotone),
//   so the candidate can neither win nor tie, and its square root is skipped.
template <int C>
__global__ void __launch_bounds__(256) k_gb_arrows(GBuild b) {
    const int nc = b.nc;
    const double half = __dmul_rn(0.5, b.d);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const double xi = b.x[i], yi = b.y[i];
        const int cxi = cell_coord(xi, b.inv_a, nc), cyi = cell_coord(yi, b.inv_a, nc);
        const double fx = __dsub_rn(xi, __dmul_rn((double)cxi, b.a));
        // corridors that may hold a disk (one bin of margin on each side)
        bool play[3];
        const float yf = __double2float_rn(yi);
        play[0] = band_count(b, yf - b.half_f - b.wf, yf + b.half_f + b.wf) > 1;  // i is there
        play[1] = band_count(b, yf + b.half_f - b.wf, yf + b.d_f + b.wf) > 0;
        play[2] = band_count(b, yf - b.d_f - b.wf, yf - b.half_f + b.wf) > 0;
        unsigned long long bt[3] = {INF_BITS, INF_BITS, INF_BITS};
        uint32_t bj[3] = {NONE, NONE, NONE};
        double bb[3] = {0.0, 0.0, 0.0};
        int rows[3] = {cyi - 1, cyi, cyi + 1};
        if (rows[0] < 0) rows[0] += nc;
        if (rows[2] >= nc) rows[2] -= nc;
        for (int m = 0; m < nc; ++m) {
            if (m >= 1) {
                unsigned long long worst = 0ull;
                bool any = false;
#pragma unroll
                for (int kc = 0; kc < 3; ++kc)
                    if (play[kc]) {
                        any = true;
                        if (bt[kc] > worst) worst = bt[kc];
                    }
                if (!any) break;
                if (worst != INF_BITS) {
                    const double thr =
                        __dsub_rn(__dsub_rn(__dmul_rn((double)m, b.a), fx), b.d);
                    const double lim = __dadd_rn(__longlong_as_double((long long)worst), b.eps);
                    if (!dneg(thr) && dbits(thr) > dbits(lim)) break;
                }
            }
            int col = cxi + m;
            if (col >= nc) col -= nc;
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                const uint32_t cell = (uint32_t)rows[rr] * (uint32_t)nc + (uint32_t)col;
                for (int sl = 0; sl < C; ++sl) {
                    const uint32_t loc = cell * C + sl;
                    const uint32_t id = b.cid[loc];
                    if (id == EMPTY) break;  // a cell's slots fill from the first
                    if (id == (uint32_t)i) continue;
                    const float ayf0 = fabsf(__fsub_rn(b.cyf[loc], yf));
                    if (fminf(ayf0, __fsub_rn(b.Lf, ayf0)) > b.dcut_f) continue;
                    const double dy = __dsub_rn(b.cy[loc], yi);
                    double ay = fabs(dy);
                    bool flip = false;
                    const double la = __dsub_rn(b.L, ay);
                    if (dbits(la) < dbits(ay)) {
                        ay = la;
                        flip = true;
                    }
                    if (dbits(ay) >= dbits(b.d)) continue;
                    int kc = 0;
                    if (dbits(ay) >= dbits(half)) {
                        bool up = !dneg(dy) && dbits(dy) != 0ull;
                        if (flip) up = !up;
                        kc = up ? 1 : 2;
                    }
                    // selects, not indexing, keep the corridor arrays in registers
                    const bool pk = kc == 0 ? play[0] : kc == 1 ? play[1] : play[2];
                    if (!pk) continue;
                    const unsigned long long bk = kc == 0 ? bt[0] : kc == 1 ? bt[1] : bt[2];
                    double dx = __dsub_rn(b.cx[loc], xi);
                    if (dneg(dx)) dx = __dadd_rn(dx, b.L);
                    const double lo = __dsub_rn(dx, b.d);
                    if (!dneg(lo) && dbits(lo) > bk) continue;
                    const double bv = __dsqrt_rn(__dsub_rn(b.d2, __dmul_rn(ay, ay)));
                    double tau = __dsub_rn(dx, bv);
                    if (dneg(tau)) tau = 0.0;
                    const unsigned long long kt = dbits(tau);
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (q == kc && (kt < bt[q] || (kt == bt[q] && id < bj[q]))) {
                            bt[q] = kt;
                            bj[q] = id;
                            bb[q] = bv;
                        }
                }
            }
        }
        GDisk &r = b.g[i];
        r.x = xi;
        r.t = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            r.a[q] = bj[q];
            r.b[q] = bj[q] == NONE ? 0.0 : bb[q];
        }
        r.pad0 = r.pad1 = 0;
    }
}

// Owner words and claims from scratch: every disk static, then the chains'
// start disks active.
__global__ void k_g_init(GDev s) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < s.n) {
        s.g[q].own = OWN_STATIC;
        s.claim[q] = 0u;
    }
}

__global__ void k_g_init_chains(GDev s, const int32_t *active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.k) return;
    const uint32_t a = (uint32_t)active[c];
    s.ci[c] = a;
    s.ci0[c] = a;
    s.g[a].own = OWN_ACTIVE | (uint32_t)c;
    s.nrec[c] = 0;
    s.status[c] = ST_STALLED;
}


// --------------------------------------------------------------- one step

// Another chain's active or stalled disk among the arrow targets of disk i
// (record r, with b): in a run of Alg. 4 it stops chain i (Remark 10) only if
// i could reach it within its remaining length D; beyond D it matters only
// through Eq. 2 (t_i + tau > t_j), which must still hold.
__device__ __forceinline__ bool active_in_reach(const GDisk &r, double b, double xi, double ti,
                                                double D, double L) {
    double dx = __dsub_rn(r.x, xi);
    if (dneg(dx)) dx = __dadd_rn(dx, L);
    double tau = __dsub_rn(dx, b);
    if (dneg(tau)) tau = 0.0;
    if (dbits(tau) < dbits(D)) return true;
    return !(dbits(__dadd_rn(ti, tau)) > dbits(r.t));
}

// What one step found.
struct GStep {
    double tau;        // tau* (lift) or D (stall)
    uint32_t j;        // target (lift)
    int lift;
    double xj, tj;     // the target's x and local time as read
    int conflict;      // a disk read is held by a chain of the other side
    uint32_t partner;  // that chain
    int viol;          // a static target fails Eq. 2 (t_i + tau > t_j, strict)
    int nonstatic;     // a target is another chain's active or stalled disk in reach ...
    uint32_t ns_owner; // ... of this chain (the first such target)
    GDisk jr;          // the target's record as read: its arrows serve the next step
};

// Is chain h, which holds a claim a repair step met, on the repairing side?
// Yes if this round's component lists it (memb == tag); with adopt, also if
// it was, or now is, taken over: a chain in no component of this round whose
// events are final since the round began joins the component (and any later
// merge that reaches the component takes it along).
__device__ __forceinline__ bool holder_ours(const GDev &s, int h, int root, uint64_t tag,
                                            bool adopt) {
    if (h < 0 || h >= s.k) return false;
    if (__ldcg((const unsigned long long *)s.memb + h) == tag) return true;
    if (!adopt) return false;
    int hc = __ldcg(s.comp_of + h);
    if (hc == h && h != root && __ldcg(s.fin + h) == 1) {
        const int prev = atomicCAS(s.comp_of + h, h, root);
        if (prev == h) {
            uf_union(s.uf, h, root);
            hc = root;
        } else {
            hc = prev;
        }
    }
    return hc == root;
}

// The next event of chain c (Sec. 2.2) along the arrows a[] (with b[]) of
// its active disk i at x_i, t_i, with remaining length D. Every disk read is
// claimed for the window (atomicCAS of the disk's claim word from 0 to c + 1,
// issued together with the loads; what was read is used only once the claims
// stand): i itself when claim_i, and each arrow target. A claim held by
// another chain is a conflict unless that chain is listed in this round's
// component (memb == tag). adopt (continuation): a holder in no component of
// this round, whose events are final since the round began, is taken over by
// the component (it joins it for any later merge) instead of being a conflict;
// the replay that a failed continuation falls back to does not count such
// chains as members, so it meets them and merges them next round.
// Candidates are the static targets (Alg. 2: j not active); a target with
// t_i + tau < t_j became static after chain c's disk had passed it and is one
// lap away (lazy per-chain frame); ties go to the lower disk index.
__device__ GStep graph_step(const GDev &s, int c, int root, uint64_t tag, const uint32_t a[3],
                            const double b[3], uint32_t i, double xi, double ti, double D,
                            bool claim_i, bool adopt = false) {
    const uint32_t mine = (uint32_t)c + 1u;
    uint32_t old[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (a[q] != NONE) old[q] = atomicCAS(s.claim + a[q], 0u, mine);
    if (claim_i) old[3] = atomicCAS(s.claim + i, 0u, mine);
    GDisk r[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (a[q] != NONE) r[q] = s.g[a[q]];
    GStep o;
    o.conflict = 0;
    o.partner = NONE;
    o.viol = 0;
    o.nonstatic = 0;
    o.ns_owner = NONE;
    // time of flight to each static target (Sec. 2.2): forward image in x,
    // b_ij fixed with the arrow, clamped at 0
    unsigned long long bt = INF_BITS;
    int bq = -1;
    uint32_t bjid = NONE;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (a[q] == NONE) continue;
        if (r[q].own != OWN_STATIC) {
            if (!o.nonstatic && active_in_reach(r[q], b[q], xi, ti, D, s.L)) {
                o.ns_owner = r[q].own & OWN_CHAIN;
                o.nonstatic = 1;
            }
            continue;
        }
        double dx = __dsub_rn(r[q].x, xi);
        if (dneg(dx)) dx = __dadd_rn(dx, s.L);
        double tau = __dsub_rn(dx, b[q]);
        if (dneg(tau)) tau = 0.0;
        if (dbits(r[q].t) != 0ull) {
            const double sum = __dadd_rn(ti, tau);
            if (!(dbits(sum) > dbits(r[q].t))) o.viol = 1;
            if (dbits(sum) < dbits(r[q].t)) tau = __dadd_rn(tau, s.L);
        }
        const unsigned long long tb = dbits(tau);
        if (bq < 0 || tb < bt || (tb == bt && a[q] < bjid)) {
            bt = tb;
            bq = q;
            bjid = a[q];
        }
    }
    // the claims: a taken one names the chain that holds the disk
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t w = old[q];
        if (w == 0u || w == mine) continue;
        const int h = (int)w - 1;
        if (holder_ours(s, h, root, tag, adopt)) continue;
        if (!o.conflict) {
            o.conflict = 1;
            o.partner = (uint32_t)h;
        }
    }
    if (bq >= 0 && bt < dbits(D)) {
        o.lift = 1;
        o.tau = __longlong_as_double((long long)bt);
        o.j = bjid;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q == bq) o.jr = r[q];  // a select, not an indexed (local-memory) load
        o.xj = o.jr.x;
        o.tj = o.jr.t;
    } else {
        o.lift = 0;
        o.tau = D;
        o.j = NONE;
        o.xj = o.tj = 0.0;
    }
    return o;
}

// Executes chain c's step from disk i (a lifting, Eq. 1, or a stall at the
// breakpoint) and writes its record at index nr (the caller checked the
// capacity and counts records and liftings).
__device__ void graph_apply(const GDev &s, int c, uint32_t i, double xi, double ti, double D,
                            int lift, uint32_t j, double tau, double xj, double tj,
                            uint32_t seq, int32_t nr) {
    GEv u;
    u.i = i;
    u.seq = seq;
    u.pad = 0;
    u.x_old = xi;
    u.ti_old = ti;
    GDisk &ri = s.g[i];
    if (lift) {
        const double tnew = __dadd_rn(ti, tau);       // new t_j = new t_i (before x, Remark 11)
        const double xnew = wrap_add(xi, tau, s.L);   // i moves to contact
        GDisk &rj = s.g[j];
        rj.own = OWN_ACTIVE | (uint32_t)c;             // j active (the claim holds j)
        rj.t = tnew;
        ri.t = tnew;
        ri.x = xnew;
        ri.own = OWN_STATIC;                           // i static
        u.j = j;
        u.tj_old = tj;
        u.t = tnew;
        u.tau = tau;
        u.xi = xnew;
        u.xj = xj;
        u.d_after = __dsub_rn(D, tau);                 // remaining length
    } else {
        const double tnew = __dadd_rn(ti, D);         // t_i reaches the breakpoint
        const double xnew = wrap_add(xi, D, s.L);     // i moves by D
        ri.x = xnew;
        ri.t = tnew;
        ri.own = OWN_STALLED | (uint32_t)c;           // stalled
        u.j = NONE;
        u.tj_old = 0.0;
        u.t = tnew;
        u.tau = D;
        u.xi = xnew;
        u.xj = 0.0;
        u.d_after = 0.0;                              // no length left
    }
    *grec_at(s, c, nr) = u;
}

// ------------------------------------------------------------------ legs

// Leg start: clear the local times the previous leg wrote (every disk its
// records name), then start every chain on its stalled disk with D = ell.
__device__ void g_leg_begin_chain(const GDev &s, int c) {
    const int32_t nr = s.nrec[c];
    // in batches: the record loads of a batch are issued before its stores
    for (int32_t e0 = 0; e0 < nr; e0 += 8) {
        uint32_t ii[8], jj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            ii[u] = e0 + u < nr ? grec_at(s, c, e0 + u)->i : NONE;
            jj[u] = e0 + u < nr ? grec_at(s, c, e0 + u)->j : NONE;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (ii[u] != NONE) s.g[ii[u]].t = 0.0;
            if (jj[u] != NONE) s.g[jj[u]].t = 0.0;
        }
    }
    const uint32_t i = s.ci[c];
    s.g[i].own = OWN_ACTIVE | (uint32_t)c;
    s.ci0[c] = i;
    s.D[c] = s.ell;
    s.tc[c] = 0.0;
    s.status[c] = ST_RUNNING;
    s.partner[c] = -1;
    s.nrec[c] = 0;
    s.nlift[c] = 0;
}

// Parallel pass of a claim window [tw, tend): one thread runs chain c from
// its state through its events before tend, until it stalls, pauses at tend
// or meets another chain: a claim it holds, or its active or stalled disk
// among the arrow targets within reach (the step is then not taken; cf.
// Remark 10). Once a
// step's winner j is known (and the step will be taken unless a claim of it
// fails), the arrow targets of j are claimed and their records loaded into
// registers, so that the next step's trips overlap this step's wait and
// writes (an L1 prefetch measured no better than a plain L2 load). Those
// disks belong to the chain's run alone, so the claims change no flag.
__device__ __noinline__ void g_pass1_chain(const GDev &s, int c, double tw, double tend) {
    if (s.status[c] != ST_RUNNING) return;
    const uint32_t mine = (uint32_t)c + 1u;
    uint32_t i = s.ci[c];
    const GDisk ri = s.g[i];
    if (ri.own != (OWN_ACTIVE | (uint32_t)c)) gdiag(s, 6, tw, c, i, ri.own, 0, 0);
    uint32_t a[3] = {ri.a[0], ri.a[1], ri.a[2]};
    double b[3] = {ri.b[0], ri.b[1], ri.b[2]};
    double xi = ri.x, ti = s.tc[c], D = s.D[c];
    int32_t nr = s.nrec[c];
    bool conflict = false;
    uint32_t partner = NONE;
    auto meet = [&](uint32_t h) {
        if (!conflict) {
            conflict = true;
            partner = h;
        }
    };
    // the first step of the window claims the active disk too
    uint32_t old[3] = {0u, 0u, 0u};
    {
        const uint32_t oi = atomicCAS(s.claim + i, 0u, mine);
        if (oi != 0u && oi != mine) meet(oi - 1u);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (a[q] != NONE) old[q] = atomicCAS(s.claim + a[q], 0u, mine);
    }
    int st = ST_RUNNING;
    bool blocked = false;
    uint32_t lifts = 0;
    GDisk r[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (a[q] != NONE) r[q] = s.g[a[q]];
    for (;;) {
        // time of flight and (tau, j) minimum over the static targets (see graph_step)
        unsigned long long bt = INF_BITS;
        int bq = -1;
        uint32_t bjid = NONE, ns_owner = NONE;
        bool hz = false;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (a[q] == NONE) continue;
            if (r[q].own != OWN_STATIC) {
                if (ns_owner == NONE && active_in_reach(r[q], b[q], xi, ti, D, s.L))
                    ns_owner = r[q].own & OWN_CHAIN;
                continue;
            }
            double dx = __dsub_rn(r[q].x, xi);
            if (dneg(dx)) dx = __dadd_rn(dx, s.L);
            double tau = __dsub_rn(dx, b[q]);
            if (dneg(tau)) tau = 0.0;
            if (dbits(r[q].t) != 0ull) {
                const double sum = __dadd_rn(ti, tau);
                if (dbits(sum) < dbits(r[q].t)) {
                    if (dbits(r[q].t) >= dbits(tw)) hz = true;
                    tau = __dadd_rn(tau, s.L);
                }
            }
            const unsigned long long tb = dbits(tau);
            if (bq < 0 || tb < bt || (tb == bt && a[q] < bjid)) {
                bt = tb;
                bq = q;
                bjid = a[q];
            }
        }
        const int lift = bq >= 0 && bt < dbits(D);
        GDisk wr;  // the winner's record, by select (no indexed local-memory access)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q == bq) wr = r[q];
        const double tau = lift ? __longlong_as_double((long long)bt) : D;
        const double T = __dadd_rn(ti, tau);
        const bool go = dbits(T) < dbits(tend) && ns_owner == NONE;
        // the next step's claims and records, requested before this step's
        // claims are resolved
        uint32_t oldn[3] = {0u, 0u, 0u};
        GDisk rn[3];
        if (lift && go) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (wr.a[q] != NONE) {
                    oldn[q] = atomicCAS(s.claim + wr.a[q], 0u, mine);
                    rn[q] = s.g[wr.a[q]];
                }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (old[q] != 0u && old[q] != mine) meet(old[q] - 1u);
        if (!conflict && ns_owner != NONE) meet(ns_owner);
        if (conflict) {
            blocked = true;
            break;
        }
        // Eq. 2 on the disks of this window: cannot fail while
        // they are held by a lone chain; an assertion
        if (hz) atomicAdd(s.lc + LC_HORIZON, 1ull);
        if (!go) break;  // pauses at the window end
        if (dbits(T) < dbits(tw)) {
            atomicAdd(s.lc + LC_ORDER, 1ull);
            gdiag(s, 9, tw, c, i, lift ? bjid : NONE, ti, tau);
        }
        if (nr >= s.cap) {
            atomicAdd(s.lc + LC_ERR_REC, 1ull);
            blocked = true;
            partner = NONE;
            break;
        }
        const uint32_t j = lift ? bjid : NONE;
        graph_apply(s, c, i, xi, ti, D, lift, j, tau, lift ? wr.x : 0.0, lift ? wr.t : 0.0,
                    (uint32_t)nr, nr);
        ++nr;
        if (!lift) {
            st = ST_STALLED;
            xi = wrap_add(xi, D, s.L);
            ti = T;
            D = 0.0;
            break;
        }
        ++lifts;
        xi = wr.x;
        i = j;
        ti = T;
        D = __dsub_rn(D, tau);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            a[q] = wr.a[q];
            b[q] = wr.b[q];
            old[q] = oldn[q];
            r[q] = rn[q];
        }
    }
    if (blocked) st = ST_BLOCKED;
    // events before the blocking time, and all before the window, are exact
    s.vt[c] = blocked ? fmax(ti, tw) : INFINITY;
    s.partner[c] = blocked && partner < (uint32_t)s.k ? (int32_t)partner : -1;
    s.status[c] = st;
    s.ci[c] = i;
    s.tc[c] = ti;
    s.D[c] = D;
    s.nrec[c] = nr;
    s.nlift[c] += (int32_t)lifts;
    if (blocked) {
        atomicAdd(s.lc + LC_BLOCKED, 1ull);
        atomicAdd(s.lc + LC_WBLOCKED, 1ull);
    }
    if (lifts) atomicAdd(s.lc + LC_P1LIFTS, (unsigned long long)lifts);
}

// --------------------------------------------------------------- repairs

// Exact inverse of graph_apply for one record of chain c.
__device__ void g_undo(const GDev &s, int c, const GEv &u) {
    GDisk &ri = s.g[u.i];
    ri.x = u.x_old;
    ri.t = u.ti_old;
    ri.own = OWN_ACTIVE | (uint32_t)c;
    if (u.j != NONE) {
        GDisk &rj = s.g[u.j];
        rj.t = u.tj_old;
        rj.own = OWN_STATIC;
        s.nlift[c] -= 1;
    }
}

// Rolls the members of a component back to T* (their events before T* are
// exact): records with event time >= T* are undone, latest first. Records of
// repair rounds (seq >= REPAIR_SEQ0) may touch one disk from several members
// and are undone one at a time in descending seq; beneath them, the records
// of the window's parallel pass touch disks claimed by their own chain only,
// so each member undoes its own in parallel.
__device__ void g_rollback(const GDev &s, const int32_t *mem, int m, double Ts) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t bseq = 0;
        int bmem = -1;
        for (int e = lane; e < m; e += 32) {
            const int c = mem[e];
            const int32_t nr = s.nrec[c];
            if (nr == 0) continue;
            const GEv &u = *grec_at(s, c, nr - 1);
            if (!(u.t >= Ts) || u.seq < REPAIR_SEQ0) continue;
            if (bmem < 0 || u.seq > bseq || (u.seq == bseq && e < bmem)) {
                bseq = u.seq;
                bmem = e;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t s2 = __shfl_xor_sync(FULL, bseq, o);
            const int m2 = __shfl_xor_sync(FULL, bmem, o);
            if (m2 >= 0 && (bmem < 0 || s2 > bseq || (s2 == bseq && m2 < bmem))) {
                bseq = s2;
                bmem = m2;
            }
        }
        if (bmem < 0) break;
        if (lane == 0) {
            const int c = mem[bmem];
            const int32_t nr = s.nrec[c];
            g_undo(s, c, *grec_at(s, c, nr - 1));
            s.nrec[c] = nr - 1;
        }
        __syncwarp();
    }
    for (int e = lane; e < m; e += 32) {
        const int c = mem[e];
        int32_t nr = s.nrec[c];
        while (nr > 0) {
            const GEv &u = *grec_at(s, c, nr - 1);
            if (!(u.t >= Ts)) break;
            g_undo(s, c, u);
            --nr;
        }
        s.nrec[c] = nr;
    }
    __syncwarp();
}

// State of chain c after its last kept record (or at the leg start).
__device__ void g_resume(const GDev &s, int c) {
    const int32_t nr = s.nrec[c];
    if (nr == 0) {
        s.ci[c] = s.ci0[c];
        s.tc[c] = 0.0;
        s.D[c] = s.ell;
        s.status[c] = ST_RUNNING;
        return;
    }
    const GEv &u = *grec_at(s, c, nr - 1);
    if (u.j == NONE) {
        s.ci[c] = u.i;
        s.tc[c] = u.t;
        s.D[c] = 0.0;
        s.status[c] = ST_STALLED;
    } else {
        s.ci[c] = u.j;
        s.tc[c] = u.t;
        s.D[c] = u.d_after;
        s.status[c] = ST_RUNNING;
    }
}

// Pending event of member c (one thread), kept with the arrows it read.
__device__ __noinline__ void g_compute(const GDev &s, int c, int root, uint64_t tag, bool &abort,
                                       int &met) {
    const uint32_t i = s.ci[c];
    const GDisk ri = s.g[i];
    const double ti = s.tc[c], D = s.D[c];
    const GStep o = graph_step(s, c, root, tag, ri.a, ri.b, i, ri.x, ti, D, true);
    if (o.conflict && !abort) {
        abort = true;
        met = (int)o.partner;
    }
    s.ev_T[c] = __dadd_rn(ti, o.tau);
    s.ev_tau[c] = o.tau;
    s.ev_j[c] = o.j;
    s.ev_lift[c] = o.lift;
    s.ev_xj[c] = o.xj;
    s.ev_tj[c] = o.tj;
#pragma unroll
    for (int q = 0; q < 3; ++q) s.ev_a[3 * (size_t)c + q] = ri.a[q];
}

// Restart mode: chain c back to time Ts. Its records at or after Ts are all
// of the current pass, whose disks each chain held alone, so every chain
// undoes its own (latest first) in parallel with the others.
__device__ void g_rollback_chain(const GDev &s, int c, double Ts) {
    int32_t nr = s.nrec[c];
    while (nr > 0) {
        const GEv &u = *grec_at(s, c, nr - 1);
        if (!(u.t >= Ts)) break;
        g_undo(s, c, u);
        --nr;
    }
    s.nrec[c] = nr;
    g_resume(s, c);
}

// After a component's replay: record abort or success for the next round.
// keep_vt (success by continuation): the members' vt becomes `now` instead of
// infinity, so that a later merge rolls them back to `now` or earlier (their
// events were applied chain by chain, not in time order).
__device__ void g_finish(const GDev &s, const int32_t *mem, int m, int root, bool abort,
                         int met, double now, int round, bool keep_vt = false) {
    const int lane = threadIdx.x & 31;
    if (abort) {
        // events before `now` are exact; the chain met joins next round
        for (int e = lane; e < m; e += 32) s.vt[mem[e]] = now;
        if (lane == 0) {
            if (met >= 0 && met < s.k) {
                s.abort_to[root] = met;
                atomic_min_time(s.vt + met, now);
            }
            atomicAdd(s.nabort + (round & 1), 1);
        }
    } else {
        for (int e = lane; e < m; e += 32) {
            s.fin[mem[e]] = 2;
            s.vt[mem[e]] = keep_vt ? now : INFINITY;
        }
    }
    __syncwarp();
}

// First repair round of a window: the blocked members continue from where
// they stopped, one after another (lane 0), over the state the others left.
// The parallel pass was a run of Alg. 4 in which every chain read only disks
// it held, every step satisfied the horizon condition and no step was taken
// towards another chain's active disk. If every continued step satisfies
// Eq. 2 on each arrow target as well, the whole is a run of Alg. 4 without a
// horizon violation, which by Lemma 2 ends where Alg. 2 ends: nothing has to
// be redone. A chain that finds the active disk of another blocked member
// among its arrow targets waits (Remark 10) while that member continues
// first. Otherwise the caller rolls the component back to T* and replays it
// in global order.
enum { CONT_DONE = 0, CONT_FAIL = 1, CONT_FOREIGN = 2 };

__device__ __noinline__ int g_continue(const GDev &s, const int32_t *mem, int m, int root,
                                       uint64_t tag, int round, double tw, double tend,
                                       int *met) {
    const int lane = threadIdx.x & 31;
    int how = CONT_DONE, who = -1;
    if (lane == 0) {
        uint32_t cnt = 0;
        int switches = 0;
        int e = 0;
        int cur = -1;
        int known = -1;  // a holder already found on this side
        while (how == CONT_DONE) {
            if (cur < 0) {  // the next member still blocked
                while (e < m && s.status[mem[e]] != ST_BLOCKED) ++e;
                if (e >= m) break;
                cur = mem[e];
            }
            const int c = cur;
            const uint32_t mine = (uint32_t)c + 1u;
            uint32_t i = s.ci[c];
            const GDisk ri = s.g[i];
            uint32_t a[3] = {ri.a[0], ri.a[1], ri.a[2]};
            double b[3] = {ri.b[0], ri.b[1], ri.b[2]};
            double xi = ri.x, ti = s.tc[c], D = s.D[c];
            int32_t nr = s.nrec[c], nl = 0;
            int st = ST_RUNNING, next = -1;
            // claims of the active disk (first step) and of the arrow targets
            uint32_t oi = atomicCAS(s.claim + i, 0u, mine);
            uint32_t old[3] = {0u, 0u, 0u};
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (a[q] != NONE) old[q] = atomicCAS(s.claim + a[q], 0u, mine);
            auto ours = [&](uint32_t w) {
                if (w == 0u || w == mine) return true;
                const int h = (int)w - 1;
                if (h == known) return true;
                if (!holder_ours(s, h, root, tag, true)) {
                    who = h;
                    return false;
                }
                known = h;
                return true;
            };
            for (;;) {
                GDisk r[3];
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (a[q] != NONE) r[q] = s.g[a[q]];
                unsigned long long bt = INF_BITS;
                int bq = -1;
                uint32_t bjid = NONE, ns_owner = NONE;
                bool viol = false;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (a[q] == NONE) continue;
                    if (r[q].own != OWN_STATIC) {
                        if (ns_owner == NONE && active_in_reach(r[q], b[q], xi, ti, D, s.L))
                            ns_owner = r[q].own & OWN_CHAIN;
                        continue;
                    }
                    double dx = __dsub_rn(r[q].x, xi);
                    if (dneg(dx)) dx = __dadd_rn(dx, s.L);
                    double tau = __dsub_rn(dx, b[q]);
                    if (dneg(tau)) tau = 0.0;
                    // Eq. 2, strict (a lap-away target fails it too)
                    if (dbits(r[q].t) != 0ull && !(dbits(__dadd_rn(ti, tau)) > dbits(r[q].t)))
                        viol = true;
                    const unsigned long long tb = dbits(tau);
                    if (bq < 0 || tb < bt || (tb == bt && a[q] < bjid)) {
                        bt = tb;
                        bq = q;
                        bjid = a[q];
                    }
                }
                const int lift = bq >= 0 && bt < dbits(D);
                GDisk wr;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q == bq) wr = r[q];
                const double tau = lift ? __longlong_as_double((long long)bt) : D;
                const double T = __dadd_rn(ti, tau);
                const bool go = dbits(T) < dbits(tend) && !viol && ns_owner == NONE;
                uint32_t oldn[3] = {0u, 0u, 0u};
                if (lift && go) {
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (wr.a[q] != NONE) {
                            oldn[q] = atomicCAS(s.claim + wr.a[q], 0u, mine);
                            prefetch_l1(s.g + wr.a[q]);
                        }
                }
                bool foreign = !ours(oi);
#pragma unroll
                for (int q = 0; q < 3; ++q) foreign = foreign || !ours(old[q]);
                oi = 0u;
                if (foreign) {
                    how = CONT_FOREIGN;
                    break;
                }
                if (viol) {
                    how = CONT_FAIL;
                    break;
                }
                if (ns_owner != NONE) {
                    const int h = (int)ns_owner;
                    if (h != c && h >= 0 && h < s.k &&
                        __ldcg((const unsigned long long *)s.memb + h) == tag &&
                        s.status[h] == ST_BLOCKED && switches < 4 * m + 4) {
                        next = h;  // wait for that member (Remark 10)
                        st = ST_BLOCKED;
                        ++switches;
                    } else {
                        how = CONT_FAIL;
                    }
                    break;
                }
                if (!(dbits(T) < dbits(tend))) break;  // pauses at the window end
                if (dbits(T) < dbits(tw) || nr >= s.cap) {
                    how = CONT_FAIL;
                    break;
                }
                const uint32_t j = lift ? bjid : NONE;
                graph_apply(s, c, i, xi, ti, D, lift, j, tau, lift ? wr.x : 0.0,
                            lift ? wr.t : 0.0, ((uint32_t)round << 24) | cnt++, nr);
                ++nr;
                if (!lift) {
                    st = ST_STALLED;
                    ti = T;
                    D = 0.0;
                    break;
                }
                ++nl;
                i = j;
                xi = wr.x;
                ti = T;
                D = __dsub_rn(D, tau);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    a[q] = wr.a[q];
                    b[q] = wr.b[q];
                    old[q] = oldn[q];
                }
            }
            // the events so far stand (a failure rolls them back with the rest)
            s.nrec[c] = nr;
            s.nlift[c] += nl;
            if (how != CONT_DONE) break;
            s.status[c] = st;
            s.ci[c] = i;
            s.tc[c] = ti;
            s.D[c] = D;
            cur = next;
        }
    }
    how = __shfl_sync(FULL, how, 0);
    *met = __shfl_sync(FULL, who, 0);
    __syncwarp();
    return how;
}

// Component q of this round (one warp): roll its members back to T*, then
// replay them in global event-time order (Alg. 2) up to the window's end.
// Members are spread over the lanes (member e on lane e mod 32); after each
// event only the members whose arrows read a disk it changed recompute.
__device__ __noinline__ void g_repair_component(const GDev &s, int q, int round, uint32_t wr_tag,
                                                double tw,
                                   double tend) {
    const int lane = threadIdx.x & 31;
    const int root = s.comp_root[q];
    const int off = s.comp_off[q], m = s.comp_off[q + 1] - off;
    const int32_t *mem = s.comp_mem + off;
    double Ts = INFINITY;
    for (int e = lane; e < m; e += 32) Ts = fmin(Ts, s.vt[mem[e]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Ts = fmin(Ts, __shfl_xor_sync(FULL, Ts, o));
    Ts = fmax(Ts, tw);  // earlier windows are final
    if (lane == 0) atomicAdd(s.lc + LC_REPAIRED, (unsigned long long)m);
    // the members listed for this round of this window (wr_tag names both)
    const uint64_t tag = ((uint64_t)wr_tag << 32) | (uint32_t)root;
    for (int e = lane; e < m; e += 32) s.memb[mem[e]] = tag;
    __syncwarp();
    if (round == 1) {
        int met = -1;
        const int how = g_continue(s, mem, m, root, tag, round, tw, tend, &met);
        if (how == CONT_DONE) {
            if (lane == 0) atomicAdd(s.lc + LC_CONTINUED, (unsigned long long)m);
            g_finish(s, mem, m, root, false, -1, Ts, round, true);
            return;
        }
        if (how == CONT_FOREIGN) {
            // the merged component's replay rolls back to T* (all of this
            // round's events lie after it)
            g_finish(s, mem, m, root, true, met, Ts, round);
            return;
        }
    }
    g_rollback(s, mem, m, Ts);
    for (int e = lane; e < m; e += 32) g_resume(s, mem[e]);
    __syncwarp();
    bool abort = false;
    int met = -1;
    for (int e = lane; e < m; e += 32)
        if (s.status[mem[e]] == ST_RUNNING) g_compute(s, mem[e], root, tag, abort, met);
    double now = Ts;
    uint32_t cnt = 0;
    for (;;) {
        {
            const unsigned ab = __ballot_sync(FULL, abort);
            if (ab) {
                met = __shfl_sync(FULL, met, __ffs(ab) - 1);
                abort = true;
                break;
            }
        }
        unsigned long long bT = ~0ull;
        int bc = 0x7FFFFFFF, bl = lane;
        for (int e = lane; e < m; e += 32) {
            const int c = mem[e];
            if (s.status[c] != ST_RUNNING) continue;
            const unsigned long long T = dbits(s.ev_T[c]);
            if (T < bT || (T == bT && c < bc)) {
                bT = T;
                bc = c;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long T2 = shfl_xor_u64(bT, o);
            const int c2 = __shfl_xor_sync(FULL, bc, o);
            const int l2 = __shfl_xor_sync(FULL, bl, o);
            if (T2 < bT || (T2 == bT && c2 < bc)) {
                bT = T2;
                bc = c2;
                bl = l2;
            }
        }
        if (bc == 0x7FFFFFFF) break;
        if (!(bT < dbits(tend))) break;  // the rest lies in a later window
        const double Tn = __longlong_as_double((long long)bT);
        if (dbits(Tn) < dbits(now) && lane == 0) {
            atomicAdd(s.lc + LC_ORDER, 1ull);
            gdiag(s, 2, round, bc, Tn, now, Ts, m);
        }
        now = Tn;
        uint32_t ib = NONE, jb = NONE;
        int st = ST_RUNNING;
        if (lane == bl) {
            const uint32_t i = s.ci[bc];
            const double ti = s.tc[bc], D = s.D[bc];
            GStep o;
            o.lift = s.ev_lift[bc];
            o.tau = s.ev_tau[bc];
            o.j = s.ev_j[bc];
            o.xj = s.ev_xj[bc];
            o.tj = s.ev_tj[bc];
            const double xi = s.g[i].x;
            const int32_t nr = s.nrec[bc];
            if (nr >= s.cap) {
                atomicAdd(s.lc + LC_ERR_REC, 1ull);
                st = ST_BLOCKED;
            } else {
                graph_apply(s, bc, i, xi, ti, D, o.lift, o.j, o.tau, o.xj, o.tj,
                            ((uint32_t)round << 24) | cnt, nr);
                s.nrec[bc] = nr + 1;
                if (o.lift) s.nlift[bc] += 1;
                st = o.lift ? ST_RUNNING : ST_STALLED;
            }
            ib = i;
            if (st == ST_RUNNING) {
                jb = o.j;
                s.ci[bc] = o.j;
                s.tc[bc] = __dadd_rn(ti, o.tau);
                s.D[bc] = __dsub_rn(D, o.tau);
            } else if (st == ST_STALLED) {
                s.tc[bc] = __dadd_rn(ti, D);
                s.D[bc] = 0.0;
                s.status[bc] = ST_STALLED;
            }
        }
        ++cnt;
        st = __shfl_sync(FULL, st, bl);
        ib = __shfl_sync(FULL, ib, bl);
        jb = __shfl_sync(FULL, jb, bl);
        __syncwarp();
        if (st == ST_BLOCKED) {  // out of records: reported by the host
            abort = true;
            met = -1;
            break;
        }
        for (int e = lane; e < m; e += 32) {
            const int c = mem[e];
            if (s.status[c] != ST_RUNNING) continue;
            bool redo = c == bc;
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) {
                const uint32_t v = s.ev_a[3 * (size_t)c + k2];
                redo |= v != NONE && (v == ib || v == jb);
            }
            if (redo) g_compute(s, c, root, tag, abort, met);
        }
        __syncwarp();
    }
    g_finish(s, mem, m, root, abort, met, now, round);
}

// Leg end: totals, and the lifting log (chain by chain).
__device__ void g_leg_end_chain(const GDev &s, int c, int32_t leg) {
    const int32_t nl = s.nlift[c];
    atomicAdd(s.lc + LC_LIFTS, (unsigned long long)nl);
    if (s.log_on && nl > 0) {
        const unsigned long long base = atomicAdd(s.tc_cnt + TC_LOG_N, (unsigned long long)nl);
        unsigned long long w = base;
        for (int32_t e = 0; e < s.nrec[c]; ++e) {
            const GEv *q = grec_at(s, c, e);
            if (q->j == NONE) continue;
            if ((int64_t)w < s.log_cap) {
                ecmc_lift_t L;
                L.leg = leg;
                L.c = c;
                L.i = (int32_t)q->i;
                L.j = (int32_t)q->j;
                L.t = q->t;
                L.tau = q->tau;
                L.xi = q->xi;
                L.xj = q->xj;
                s.log[w] = L;
            }
            ++w;
        }
    }
}

// ------------------------------------------- persistent multi-leg kernel

struct GCtl {
    int64_t budget;  // liftings for this run (0: none)
    int64_t lifts, legs, conflict_legs, repaired, continued, horizon, order_err, p1_lifts,
        repair_lifts, restarts, blocked, cwindows;
    uint8_t *flags;  // per-leg conflict flags (device) or null
    int32_t flags_cap;
    int32_t done;    // budget reached or error
    int32_t err;     // LC_ERR_* seen, or too many repair rounds
    int32_t pad;
    int64_t leg0;    // batches: legs run before this launch (lifting log)
};

enum { GPH_BEGIN = 0, GPH_PASS1, GPH_REPAIR, GPH_END, GPH_N };

struct GRun {
    GDev s;
    GCtl *ctl;
    unsigned int *bar;               // [2] grid barrier
    int32_t *err;                    // ECMC_ETIMEOUT from a barrier
    unsigned long long *phase_ns;    // [GPH_N] device time per phase (block 0 clock)
    int32_t max_legs;
    int64_t leg0;                    // legs run before this launch (lifting log)
    int64_t budget;                  // liftings of this launch after which it stops (0: none)
};

__device__ __forceinline__ double g_window_start(const GDev &s, int w) {
    return w == 0 ? 0.0 : __ddiv_rn(__dmul_rn((double)w, s.ell), (double)s.windows);
}

__device__ __forceinline__ double g_window_end(const GDev &s, int w) {
    return w + 1 >= s.windows ? INFINITY
                              : __ddiv_rn(__dmul_rn((double)(w + 1), s.ell), (double)s.windows);
}

constexpr int GRUN_THREADS = 256;
constexpr int GRUN_MIN_BLOCKS = 1;
constexpr int MAX_RESTARTS = 16;  // per leg, then the local repair takes over

// One cooperative launch runs up to max_legs legs. Per leg and claim window:
// the parallel pass (one thread per chain), then repair rounds (conflict
// components by one block, their replays by one warp each) until no component
// met another chain. Phases are separated by grid barriers whose waits are
// bounded (ECMC_ETIMEOUT).
__global__ void __launch_bounds__(GRUN_THREADS, GRUN_MIN_BLOCKS) k_run_graph(GRun R) {
    extern __shared__ int32_t uf_sm[];  // UF_SMEM_BYTES: the union-find working set
    __shared__ int warp_tot[32];
    __shared__ int tot[2];
    __shared__ int sflag;
    const GDev &s = R.s;
    const int lane = threadIdx.x & 31;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int nwarps = nthreads >> 5;
    const int gw = blockIdx.x + gridDim.x * (threadIdx.x >> 5);
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_prev = timer ? gtimer() : 0ull;
    auto mark = [&](int ph) {
        if (timer) {
            const unsigned long long t = gtimer();
            R.phase_ns[ph] += t - t_prev;
            t_prev = t;
        }
    };
    // The per-leg counters accumulate over the launch: a leg's totals are
    // differences, and every thread decides alike, after the leg's last
    // barrier, whether the launch goes on. Without an event budget the next
    // leg is begun in the same phase as this one ends.
    unsigned long long prev[LC_N];
#pragma unroll
    for (int q = 0; q < LC_N; ++q) prev[q] = 0ull;
    auto begin_leg = [&]() {
        for (int c = gt; c < s.k; c += nthreads) g_leg_begin_chain(s, c);
        for (int64_t q = gt; q < s.n; q += nthreads) s.claim[q] = 0u;
    };
    begin_leg();
    if (gt < LC_N) s.lc[gt] = 0ull;
    if (gt == 0) s.nabort[0] = s.nabort[1] = 0;
    if (!grid_sync(R.bar, R.err, &sflag)) return;
    mark(GPH_BEGIN);
    __shared__ double dmin[32];
    for (int leg = 0; leg < R.max_legs; ++leg) {
        // restart mode (one claim window): a pass that meets a conflict is cut
        // at T*, the earliest time a chain stopped -- every event before it is
        // exact (Remark 6) -- all chains are rolled back to T*, and T* becomes
        // the next breakpoint of the leg: a new pass from T* with new claims
        // (Sec. 3.4, second restart strategy). A pass that cannot progress
        // (T* at its own start), or the last one allowed, is repaired locally.
        double tw_r = 0.0;
        int sub = 0;
        for (int w = 0; w < s.windows; ++w) {
          for (;;) {
            if (w > 0) {
                // a new claim window: the claims of the last one are void
                for (int64_t q = gt; q < s.n; q += nthreads) s.claim[q] = 0u;
                if (!grid_sync(R.bar, R.err, &sflag)) return;
            }
            const double tw = s.restart ? tw_r : g_window_start(s, w);
            const double te = g_window_end(s, w);
            // one chain per warp (lane 0) while they last, warps interleaved over
            // the blocks so that the chains spread over all SMs
            for (int c = gw + nwarps * lane; c < s.k; c += nwarps * 32)
                g_pass1_chain(s, c, tw, te);
            if (!grid_sync(R.bar, R.err, &sflag)) return;
            mark(GPH_PASS1);
            if (s.restart) {
                if (*(volatile unsigned long long *)(s.lc + LC_WBLOCKED) == 0ull) break;
                if (blockIdx.x == 0) {  // T*: the earliest stop of this pass
                    double m = INFINITY;
                    for (int c = threadIdx.x; c < s.k; c += blockDim.x)
                        if (s.status[c] == ST_BLOCKED) m = fmin(m, s.vt[c]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(FULL, m, o));
                    if (lane == 0) dmin[threadIdx.x >> 5] = m;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmin(m, dmin[q]);
                        s.tstar[0] = fmax(m, tw);
                    }
                    __syncthreads();
                }
                if (!grid_sync(R.bar, R.err, &sflag)) return;
                const double Ts = *(volatile double *)s.tstar;
                if (!(dbits(Ts) > dbits(tw)) || sub >= MAX_RESTARTS) {
                    // no progress: the local repair below
                } else {
                    // every thread has read the blocked count: reset for the next pass
                    if (gt == 0) {
                        s.lc[LC_WBLOCKED] = 0ull;
                        s.lc[LC_RESTARTS] += 1ull;
                        if (sub == 0) s.lc[LC_CWINDOWS] += 1ull;  // the window's flag
                    }
                    for (int c = gt; c < s.k; c += nthreads) g_rollback_chain(s, c, Ts);
                    for (int64_t q = gt; q < s.n; q += nthreads) s.claim[q] = 0u;
                    if (!grid_sync(R.bar, R.err, &sflag)) return;
                    tw_r = Ts;
                    ++sub;
                    continue;
                }
            }
            if (gt == 0) s.nabort[1] = 0;  // the first round's abort count
            for (int round = 1;; ++round) {
                if (blockIdx.x == 0) {
                    const bool need = round == 1 ? s.lc[LC_WBLOCKED] != 0ull
                                                 : s.nabort[(round - 1) & 1] != 0;
                    __syncthreads();
                    if (round == 1 && threadIdx.x == 0) {
                        s.lc[LC_WBLOCKED] = 0ull;
                        if (need && sub == 0) s.lc[LC_CWINDOWS] += 1ull;
                    }
                    if (need && round <= 255) {
                        uf_block(s, round == 1, warp_tot, tot, false, uf_sm);
                    } else if (threadIdx.x == 0) {
                        s.ctl[CTL_NCOMP] = 0;
                        if (need) atomicAdd(s.lc + LC_ERR_CAP, 1ull);  // too many rounds
                    }
                    __syncthreads();
                }
                if (!grid_sync(R.bar, R.err, &sflag)) return;
                // every block has read the previous round's abort count
                if (gt == 0) s.nabort[(round + 1) & 1] = 0;
                const int ncomp = s.ctl[CTL_NCOMP];
                if (ncomp == 0) break;
                for (;;) {
                    int q = 0;
                    if (lane == 0) q = atomicAdd(s.ctl + CTL_WORK, 1);
                    q = __shfl_sync(FULL, q, 0);
                    if (q >= ncomp) break;
                    g_repair_component(s, q, round,
                                       ((uint32_t)(leg * s.windows + w) << 8) | (uint32_t)round,
                                       tw, te);
                }
                if (!grid_sync(R.bar, R.err, &sflag)) return;
                // no component met another chain: the window is repaired
                if (*(volatile int32_t *)(s.nabort + (round & 1)) == 0) break;
            }
            mark(GPH_REPAIR);
            break;
          }
        }
        // leg end: liftings and the log (and, without a budget, the next leg's
        // start), then the totals. Every counter but the liftings is final
        // since the last barrier (the next leg's pass may start as soon as the
        // coming barrier is passed), so thread 0 takes them now.
        const volatile unsigned long long *lcv = s.lc;
        // errors of this leg are final too: all threads read them here, so
        // that they all take the same decision below
        const bool err = lcv[LC_ERR_REC] != 0ull || lcv[LC_ERR_CAP] != 0ull;
        unsigned long long d[LC_N];
        if (gt == 0) {
#pragma unroll
            for (int q = 0; q < LC_N; ++q) {
                if (q == LC_LIFTS) continue;
                const unsigned long long v = lcv[q];
                d[q] = v - prev[q];
                prev[q] = v;
            }
        }
        const bool more = leg + 1 < R.max_legs && R.budget == 0;
        for (int c = gt; c < s.k; c += nthreads) {
            g_leg_end_chain(s, c, (int32_t)(R.leg0 + leg));
            if (more) g_leg_begin_chain(s, c);
        }
        if (more)
            for (int64_t q = gt; q < s.n; q += nthreads) s.claim[q] = 0u;
        if (!grid_sync(R.bar, R.err, &sflag)) return;
        // (read by all threads; with a budget no next leg has begun)
        const unsigned long long lifts_all = lcv[LC_LIFTS];
        if (gt == 0) {
            GCtl &c = *R.ctl;
            d[LC_LIFTS] = lifts_all - prev[LC_LIFTS];
            prev[LC_LIFTS] = lifts_all;
            const int flag = d[LC_BLOCKED] != 0ull;
            if (c.flags && c.legs < c.flags_cap) c.flags[c.legs] = (uint8_t)flag;
            c.lifts += (int64_t)d[LC_LIFTS];
            c.p1_lifts += (int64_t)d[LC_P1LIFTS];
            if (flag) c.repair_lifts += (int64_t)d[LC_LIFTS];
            c.legs += 1;
            c.conflict_legs += flag;
            c.repaired += (int64_t)d[LC_REPAIRED];
            c.continued += (int64_t)d[LC_CONTINUED];
            c.restarts += (int64_t)d[LC_RESTARTS];
            c.blocked += (int64_t)d[LC_BLOCKED];
            c.cwindows += (int64_t)d[LC_CWINDOWS];
            c.horizon += (int64_t)d[LC_HORIZON];
            c.order_err += (int64_t)d[LC_ORDER];
            if (err) c.err = 1;
        }
        mark(GPH_END);
        if (err || (R.budget > 0 && (int64_t)lifts_all >= R.budget)) break;
        if (leg + 1 >= R.max_legs) break;
        if (!more) {
            begin_leg();
            if (!grid_sync(R.bar, R.err, &sflag)) return;
            mark(GPH_BEGIN);
        }
    }
}

// ------------------------------------- batches of constraint-graph systems

// Launch state of a batch: R systems (descriptors in device memory), their
// chains and conflict components flattened by prefix offsets.
struct GBatchDev {
    const GDev *S;          // [R]
    GCtl *ctl;              // [R]
    const int32_t *chain_base;  // [R + 1]
    int32_t *comp_base;     // [R + 1]
    int32_t *g;             // [GB_N]
    unsigned int *bar;      // [1] grid barrier
    int32_t *err;           // ECMC_ETIMEOUT from a barrier
    unsigned long long *phase_ns;  // [GPH_N]
    int32_t R, max_legs, windows;
    int32_t pad;
};

enum { GB_WORK = 0, GB_ANY, GB_DONE, GB_REMAIN0, GB_REMAIN1, GB_N };

// replica of flattened item f, with base[r] <= f < base[r + 1]
__device__ __forceinline__ int g_find_rep(const int32_t *base, int R, int f) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool g_rep_on(const GBatchDev &B, int r) {
    return !B.ctl[r].done;
}

// k_run_graph over R systems (the local repair; no restart mode): every
// system's legs exactly as k_run_graph computes them. Per leg and claim
// window: the parallel pass over all systems' chains (one thread per chain),
// the union-find of each system's conflict components (one block per
// system), their repairs from one work queue (one warp per component), the
// leg end and each system's totals; the launch ends when every system has
// reached max_legs or its liftings budget.
__global__ void __launch_bounds__(GRUN_THREADS, GRUN_MIN_BLOCKS) k_run_graph_batch(GBatchDev B) {
    extern __shared__ int32_t uf_sm[];
    __shared__ int warp_tot[32];
    __shared__ int tot[2];
    __shared__ int sflag;
    const int lane = threadIdx.x & 31;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int nwarps = nthreads >> 5;
    const int gw = blockIdx.x + gridDim.x * (threadIdx.x >> 5);
    const int R = B.R;
    const int total_chains = B.chain_base[R];
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_prev = timer ? gtimer() : 0ull;
    auto mark = [&](int ph) {
        if (timer) {
            const unsigned long long t = gtimer();
            B.phase_ns[ph] += t - t_prev;
            t_prev = t;
        }
    };
    // true in the last block to get here, of all blocks (each comes once per use)
    auto last_block = [&]() -> bool {
        // (as in the grid barrier: the block barrier, then the master
        // thread's fences, release before the count and acquire after it)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int old = atomicAdd(B.g + GB_DONE, 1);
            sflag = (old + 1) % (int)gridDim.x == 0;
            if (sflag) __threadfence();
        }
        __syncthreads();
        const bool last = sflag != 0;
        __syncthreads();
        return last;
    };
    for (int leg = 0; leg < B.max_legs; ++leg) {
        // leg start of every running system: chains, claims, per-leg counters
        for (int f = gt; f < total_chains; f += nthreads) {
            const int r = g_find_rep(B.chain_base, R, f);
            if (g_rep_on(B, r)) g_leg_begin_chain(B.S[r], f - B.chain_base[r]);
        }
        for (int r = 0; r < R; ++r) {
            if (!g_rep_on(B, r)) continue;
            const GDev &s = B.S[r];
            for (int64_t q = gt; q < s.n; q += nthreads) s.claim[q] = 0u;
            if (gt < LC_N) s.lc[gt] = 0ull;
            if (gt == 0) s.nabort[0] = s.nabort[1] = 0;
        }
        if (!grid_sync(B.bar, B.err, &sflag)) return;
        if (gt == 0) B.g[GB_REMAIN0 + ((leg + 1) & 1)] = 0;
        mark(GPH_BEGIN);
        for (int w = 0; w < B.windows; ++w) {
            if (w > 0) {
                for (int r = 0; r < R; ++r) {
                    if (!g_rep_on(B, r)) continue;
                    const GDev &s = B.S[r];
                    for (int64_t q = gt; q < s.n; q += nthreads) s.claim[q] = 0u;
                }
                if (!grid_sync(B.bar, B.err, &sflag)) return;
            }
            // one chain per thread, warps interleaved over the blocks
            for (int f = gw + nwarps * lane; f < total_chains; f += nwarps * 32) {
                const int r = g_find_rep(B.chain_base, R, f);
                if (!g_rep_on(B, r)) continue;
                const GDev &s = B.S[r];
                g_pass1_chain(s, f - B.chain_base[r], g_window_start(s, w), g_window_end(s, w));
            }
            if (!grid_sync(B.bar, B.err, &sflag)) return;
            mark(GPH_PASS1);
            for (int r = gt; r < R; r += nthreads)
                if (g_rep_on(B, r)) B.S[r].nabort[1] = 0;  // the first round's abort count
            for (int round = 1;; ++round) {
                for (int r = blockIdx.x; r < R; r += gridDim.x) {
                    const GDev &s = B.S[r];
                    bool need = false;
                    if (g_rep_on(B, r))
                        need = round == 1 ? s.lc[LC_WBLOCKED] != 0ull
                                          : s.nabort[(round - 1) & 1] != 0;
                    __syncthreads();
                    if (round == 1 && threadIdx.x == 0 && g_rep_on(B, r)) {
                        s.lc[LC_WBLOCKED] = 0ull;
                        if (need) s.lc[LC_CWINDOWS] += 1ull;
                    }
                    if (need && round <= 255) {
                        uf_block(s, round == 1, warp_tot, tot, false, uf_sm);
                    } else if (threadIdx.x == 0) {
                        s.ctl[CTL_NCOMP] = 0;
                        if (need) atomicAdd(s.lc + LC_ERR_CAP, 1ull);  // too many rounds
                    }
                    __syncthreads();
                }
                if (last_block()) {
                    // prefix of component counts over systems
                    const int chunk = (R + blockDim.x - 1) / blockDim.x;
                    const int lo = min(R, (int)threadIdx.x * chunk), hi = min(R, lo + chunk);
                    int sum = 0;
                    for (int r = lo; r < hi; ++r) sum += B.S[r].ctl[CTL_NCOMP];
                    int off = block_exscan(sum, warp_tot, tot);
                    for (int r = lo; r < hi; ++r) {
                        B.comp_base[r] = off;
                        off += B.S[r].ctl[CTL_NCOMP];
                    }
                    if (threadIdx.x == 0) {
                        B.comp_base[R] = tot[0];
                        B.g[GB_WORK] = 0;
                        B.g[GB_ANY] = tot[0];
                    }
                }
                if (!grid_sync(B.bar, B.err, &sflag)) return;
                // every block has read the previous round's abort counts
                for (int r = gt; r < R; r += nthreads)
                    if (g_rep_on(B, r)) B.S[r].nabort[(round + 1) & 1] = 0;
                const int ncomp = B.g[GB_ANY];
                if (ncomp == 0) break;
                for (;;) {
                    int q = 0;
                    if (lane == 0) q = atomicAdd(B.g + GB_WORK, 1);
                    q = __shfl_sync(FULL, q, 0);
                    if (q >= ncomp) break;
                    const int r = g_find_rep(B.comp_base, R, q);
                    const GDev &s = B.S[r];
                    g_repair_component(s, q - B.comp_base[r], round,
                                       ((uint32_t)(leg * B.windows + w) << 8) | (uint32_t)round,
                                       g_window_start(s, w), g_window_end(s, w));
                }
                if (!grid_sync(B.bar, B.err, &sflag)) return;
                // no component met another chain: the window is repaired
                int aborted = 0;
                for (int r = threadIdx.x; r < R; r += blockDim.x)
                    if (g_rep_on(B, r) &&
                        *(volatile int32_t *)(B.S[r].nabort + (round & 1)) != 0)
                        aborted = 1;
                if (!__syncthreads_or(aborted)) break;
            }
            mark(GPH_REPAIR);
        }
        // leg end: liftings and the log; the last block takes each system's
        // totals and budget
        for (int f = gt; f < total_chains; f += nthreads) {
            const int r = g_find_rep(B.chain_base, R, f);
            if (g_rep_on(B, r))
                g_leg_end_chain(B.S[r], f - B.chain_base[r],
                                (int32_t)(B.ctl[r].leg0 + B.ctl[r].legs));
        }
        if (last_block()) {
            for (int r = threadIdx.x; r < R; r += blockDim.x) {
                GCtl *const cp = B.ctl + r;
                GCtl c = *cp;
                if (c.done) continue;
                const unsigned long long *lcp = B.S[r].lc;
                unsigned long long lc[LC_N];
#pragma unroll
                for (int q = 0; q < LC_N; ++q) lc[q] = __ldcg(lcp + q);
                const int flag = lc[LC_BLOCKED] != 0ull;
                if (c.flags && c.legs < c.flags_cap) c.flags[c.legs] = (uint8_t)flag;
                c.lifts += (int64_t)lc[LC_LIFTS];
                c.p1_lifts += (int64_t)lc[LC_P1LIFTS];
                if (flag) c.repair_lifts += (int64_t)lc[LC_LIFTS];
                c.legs += 1;
                c.conflict_legs += flag;
                c.repaired += (int64_t)lc[LC_REPAIRED];
                c.continued += (int64_t)lc[LC_CONTINUED];
                c.blocked += (int64_t)lc[LC_BLOCKED];
                c.cwindows += (int64_t)lc[LC_CWINDOWS];
                c.horizon += (int64_t)lc[LC_HORIZON];
                c.order_err += (int64_t)lc[LC_ORDER];
                if (lc[LC_ERR_REC] != 0ull || lc[LC_ERR_CAP] != 0ull) c.err = 1;
                if (c.err || (c.budget > 0 && c.lifts >= c.budget)) c.done = 1;
                *cp = c;
                if (!c.done) atomicAdd(B.g + GB_REMAIN0 + (leg & 1), 1);
            }
        }
        if (!grid_sync(B.bar, B.err, &sflag)) return;
        mark(GPH_END);
        if (B.g[GB_REMAIN0 + (leg & 1)] == 0) break;
    }
}

// Exports positions (per disk id), local times and active disks.
__global__ void k_g_export(GDev s, double *x, double *t) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s.n) return;
    if (x) x[q] = s.g[q].x;
    if (t) t[q] = s.g[q].t;
}

__global__ void k_g_export_active(GDev s, int32_t *active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < s.k) active[c] = (int32_t)s.ci[c];
}

// Direction change: the disks' x and y are exchanged (x from y_old, y from
// x_old); the graph is then rebuilt for the new frame.
__global__ void k_g_swap_xy(GDev s, double *xnew) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s.n) return;
    const double xo = s.g[q].x;
    xnew[q] = s.y[q];
    s.y[q] = xo;
}

__global__ void k_g_reset_chains(GDev s) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.k) return;
    s.nrec[c] = 0;
    s.ci0[c] = s.ci[c];
}

}  // namespace

// ------------------------------------------------------------------ host

struct GraphCtx {
    GDev s;
    int nc = 0;
    double box = 0.0;
    cudaStream_t st = nullptr;
    std::vector<void *> allocs;
    GCtl *d_ctl = nullptr;
    unsigned int *d_bar = nullptr;
    int32_t *d_err = nullptr;
    unsigned long long *d_phase = nullptr;
    uint8_t *d_flags = nullptr;
    int32_t flags_cap = 0;
    int64_t log_legs = 0;  // legs logged so far (leg index of the log)
    int grid = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void *build_tmp[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<std::pair<void **, size_t>> pending;
    int64_t bytes = 0;  // device memory held
};

namespace {

// Device arrays of a context: requested one by one, then placed in a single
// allocation (each on a 256-byte boundary) by gcommit.
template <typename T>
int galloc(GraphCtx *g, T **ptr, size_t count, std::string &) {
    *ptr = nullptr;
    g->pending.emplace_back((void **)ptr, std::max<size_t>(count, 1) * sizeof(T));
    return 0;
}

int gcommit(GraphCtx *g, std::string &err) {
    size_t total = 0;
    for (auto &r : g->pending) total += (r.second + 255) & ~(size_t)255;
    void *base = nullptr;
    if (total) {
        if (dm_alloc(&base, total) != 0) {
            g->pending.clear();
            err = "cudaMalloc failed (graph state)";
            return ECMC_ENOMEM;
        }
        g->allocs.push_back(base);
        g->bytes += (int64_t)total;
    }
    size_t off = 0;
    for (auto &r : g->pending) {
        *r.first = (char *)base + off;
        off += (r.second + 255) & ~(size_t)255;
    }
    g->pending.clear();
    return 0;
}

// Builds the arrows (and x, t = 0) of every disk from positions x, y (device).
// Bytes of the build's scratch (kept by the context for direction changes).
static int64_t graph_build_bytes(double L, double d, int nc, int C) {
    const size_t nslot = (size_t)nc * nc * C;
    const size_t nb = (size_t)((int)std::ceil(L / (d / 128.0)) + 1);
    return (int64_t)(nslot * 4 + nslot * 8 + nslot * 8 + (nb + 1) * 4 + 8 + nslot * 4 +
                     ((nb + SCAN_TILE - 1) / SCAN_TILE) * 4);
}

int graph_build(GraphCtx *g, const double *x, const double *y, std::string &err) {
    GDev &s = g->s;
    const int nc = g->nc;
    const double a = g->box / nc;
    // slots per cell: at most 4 centres at mutual distance >= d fit in a cell
    // with a < sqrt(2) d, at most 6 for a < 1.664 d
    const int C = a < std::sqrt(2.0) * s.d * (1.0 - 1e-9) ? 4 : 8;
    GBuild b;
    b.n = s.n;
    b.nc = nc;
    b.L = s.L;
    b.d = s.d;
    b.d2 = s.d * s.d;
    b.a = a;
    b.inv_a = (double)nc / s.L;
    b.eps = std::ldexp(s.L, -30);
    b.w = s.d / 128.0;
    b.Lf = (float)s.L;
    b.wf = (float)b.w;
    b.inv_wf = 1.0f / b.wf;
    b.half_f = (float)(0.5 * s.d);
    b.d_f = (float)s.d;
    // |dy| in FP32 is off by at most 2.5 ulp of L (three roundings of values
    // below L, one of L itself): L * 1e-6 covers twice that, d * 1e-3 the
    // rounding of the cut
    b.dcut_f = (float)(s.d * (1.0 + 1e-3) + s.L * 1e-6);
    b.nb = (int)std::ceil(s.L / b.w) + 1;
    b.x = x;
    b.y = y;
    b.g = s.g;
    const size_t nslot = (size_t)nc * nc * C;
    // scratch of the build, kept by the context for the next direction change
    void **tmp = g->build_tmp;
    if (!tmp[0]) {
        if (dm_alloc(&tmp[0], nslot * 4) != 0 || dm_alloc(&tmp[1], nslot * 8) != 0 ||
            dm_alloc(&tmp[2], nslot * 8) != 0 || dm_alloc(&tmp[3], ((size_t)b.nb + 1) * 4) != 0 ||
            dm_alloc(&tmp[4], 8) != 0 || dm_alloc(&tmp[5], nslot * 4) != 0 ||
            dm_alloc(&tmp[6], (((size_t)b.nb + SCAN_TILE - 1) / SCAN_TILE) * 4) != 0) {
            for (int q = 0; q < 7; ++q) {
                dm_free(tmp[q]);
                tmp[q] = nullptr;
            }
            err = "cudaMalloc failed (graph build)";
            return ECMC_ENOMEM;
        }
        g->bytes += graph_build_bytes(s.L, s.d, nc, C);
    }
    b.cid = (uint32_t *)tmp[0];
    b.cx = (double *)tmp[1];
    b.cy = (double *)tmp[2];
    b.bins = (int32_t *)tmp[3];
    b.err = (unsigned long long *)tmp[4];
    b.cyf = (float *)tmp[5];
    cudaStream_t st = g->st;
    cudaMemsetAsync(b.cid, 0xFF, nslot * 4, st);
    cudaMemsetAsync(b.bins, 0, ((size_t)b.nb + 1) * 4, st);
    cudaMemsetAsync(b.err, 0, 8, st);
    const unsigned nblk = (unsigned)((s.n + 255) / 256);
    if (C == 4)
        k_gb_cells<4><<<nblk, 256, 0, st>>>(b);
    else
        k_gb_cells<8><<<nblk, 256, 0, st>>>(b);
    {
        const unsigned tiles = (unsigned)((b.nb + SCAN_TILE - 1) / SCAN_TILE);
        int32_t *part = (int32_t *)tmp[6];
        k_gb_tile_sums<<<tiles, 1024, 0, st>>>(b, part);
        k_gb_scan_tiles<<<tiles, 1024, 0, st>>>(b, part);
    }
    const unsigned ablk = (unsigned)((s.n + 255) / 256);  // one thread per disk
    if (C == 4)
        k_gb_arrows<4><<<ablk, 256, 0, st>>>(b);
    else
        k_gb_arrows<8><<<ablk, 256, 0, st>>>(b);
    unsigned long long overflow = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&overflow, b.err, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        err = std::string("graph build: ") + cudaGetErrorString(e);
        return ECMC_ECUDA;
    }
    if (overflow) {
        err = "more disks in a cell than it has slots (overlapping input?)";
        return ECMC_ECAPACITY;
    }
    return 0;
}

}  // namespace

// The device arrays of a graph context, requested from the pool (galloc):
// graph_create commits them, graph_plan_bytes only adds them up.
static int graph_plan(GraphCtx *g, const ecmc_params *p, std::string &err) {
    GDev &s = g->s;
    const size_t n = (size_t)p->n, k = (size_t)p->n_chains;
    int rc = 0;
    auto chk = [&](int r) {
        if (r && !rc) rc = r;
    };
    chk(galloc(g, &s.g, n, err));
    chk(galloc(g, &s.y, n, err));
    chk(galloc(g, &s.ci, k, err));
    chk(galloc(g, &s.ci0, k, err));
    chk(galloc(g, &s.D, k, err));
    chk(galloc(g, &s.tc, k, err));
    chk(galloc(g, &s.status, k, err));
    chk(galloc(g, &s.partner, k, err));
    chk(galloc(g, &s.nrec, k, err));
    chk(galloc(g, &s.nlift, k, err));
    chk(galloc(g, &s.claim, n, err));
    chk(galloc(g, &s.memb, k, err));
    chk(galloc(g, &s.tstar, 1, err));
    s.restart = (p->flags & ECMC_RESTART) ? 1 : 0;
    chk(galloc(g, &s.rec, k * (size_t)s.cap, err));
    chk(galloc(g, &s.ev_T, k, err));
    chk(galloc(g, &s.ev_tau, k, err));
    chk(galloc(g, &s.ev_xj, k, err));
    chk(galloc(g, &s.ev_tj, k, err));
    chk(galloc(g, &s.ev_j, k, err));
    chk(galloc(g, &s.ev_a, 3 * k, err));
    chk(galloc(g, &s.ev_lift, k, err));
    chk(galloc(g, &s.vt, k, err));
    chk(galloc(g, &s.uf, k, err));
    chk(galloc(g, &s.fin, k, err));
    chk(galloc(g, &s.comp_of, k, err));
    chk(galloc(g, &s.abort_to, k, err));
    chk(galloc(g, &s.comp_cnt, k, err));
    chk(galloc(g, &s.comp_off, k + 1, err));
    chk(galloc(g, &s.comp_root, k, err));
    chk(galloc(g, &s.comp_mem, k, err));
    chk(galloc(g, &s.ctl, CTL_N, err));
    chk(galloc(g, &s.nabort, 2, err));
    chk(galloc(g, &s.lc, LC_N, err));
    chk(galloc(g, &s.tc_cnt, TC_N, err));
    chk(galloc(g, &s.dbg, 16, err));
    if (s.log_on) chk(galloc(g, &s.log, (size_t)s.log_cap, err));
    chk(galloc(g, &g->d_ctl, 1, err));
    chk(galloc(g, &g->d_bar, 2, err));
    chk(galloc(g, &g->d_err, 1, err));
    chk(galloc(g, &g->d_phase, GPH_N, err));
    return rc;
}


int graph_create(const ecmc_params *p, int nc, const double *x, const double *y,
                 const int32_t *active, cudaStream_t st, GraphCtx **out, std::string &err) {
    *out = nullptr;
    if (p->n_chains > MAX_CHAINS) {
        err = "too many chains";
        return ECMC_EINVAL;
    }
    GraphCtx *g = new (std::nothrow) GraphCtx();
    if (!g) {
        err = "host allocation";
        return ECMC_ENOMEM;
    }
    g->nc = nc;
    g->box = p->box;
    g->st = st;
    GDev &s = g->s;
    memset(&s, 0, sizeof s);
    s.n = p->n;
    s.k = p->n_chains;
    s.nc = nc;
    s.cap = p->undo_cap > 0 ? p->undo_cap : 1024;
    s.windows = p->windows > 0 ? p->windows : 1;
    s.L = p->box;
    s.d = p->d;
    s.ell = p->ell;
    s.log_on = (p->flags & ECMC_LOG_LIFTINGS) ? 1 : 0;
    s.log_cap = s.log_on ? (p->log_cap > 0 ? p->log_cap : ((int64_t)1 << 22)) : 0;
    const size_t n = (size_t)p->n, k = (size_t)p->n_chains;
    int rc = 0;
    auto chk = [&](int r) {
        if (r && !rc) rc = r;
    };
    chk(graph_plan(g, p, err));
    chk(gcommit(g, err));
    if (!rc && (cudaEventCreate(&g->ev0) != cudaSuccess || cudaEventCreate(&g->ev1) != cudaSuccess)) {
        err = "event creation";
        rc = ECMC_ECUDA;
    }
    if (rc) {
        graph_destroy(g);
        return rc;
    }
    cudaMemcpyAsync(s.y, y, n * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(s.nrec, 0, k * 4, st);
    cudaMemsetAsync(s.memb, 0xFF, k * 8, st);
    cudaMemsetAsync(s.lc, 0, LC_N * 8, st);
    cudaMemsetAsync(s.tc_cnt, 0, TC_N * 8, st);
    cudaMemsetAsync(s.dbg, 0, 16 * 8, st);
    rc = graph_build(g, x, s.y, err);
    if (rc) {
        graph_destroy(g);
        return rc;
    }
    k_g_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s);
    k_g_init_chains<<<(unsigned)((k + 127) / 128), 128, 0, st>>>(s, active);
    int dev = 0, n_sm = 1, blocks = 0, coop = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_run_graph, GRUN_THREADS,
                                                          UF_SMEM_BYTES);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || !coop || blocks < 1) {
        (void)cudaGetLastError();
        err = e != cudaSuccess ? std::string("graph create: ") + cudaGetErrorString(e)
                               : std::string("cooperative launch unavailable");
        graph_destroy(g);
        return ECMC_ECUDA;
    }
    g->grid = n_sm * std::min(blocks, GRUN_MIN_BLOCKS);
    *out = g;
    return 0;
}

int graph_run(GraphCtx *g, int32_t n_legs, uint64_t budget, uint8_t *flags_host,
              int32_t *legs_done, GraphTotals *tot, std::string &err) {
    memset(tot, 0, sizeof *tot);
    if (legs_done) *legs_done = 0;
    if (n_legs <= 0) return 0;
    if ((int64_t)n_legs * g->s.windows >= ((int64_t)1 << 24)) {
        err = "too many legs x windows for one call (< 2^24)";
        return ECMC_EINVAL;
    }
    cudaStream_t st = g->st;
    if (g->flags_cap < n_legs) {
        dm_free(g->d_flags);
        g->d_flags = nullptr;
        g->flags_cap = 0;
        if (dm_alloc_t(&g->d_flags, (size_t)n_legs) != 0) {
            err = "flags allocation";
            return ECMC_ENOMEM;
        }
        g->flags_cap = n_legs;
    }
    GCtl ctl;
    memset(&ctl, 0, sizeof ctl);
    ctl.budget = (int64_t)budget;
    ctl.flags = g->d_flags;
    ctl.flags_cap = g->flags_cap;
    int rc = 0;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && !rc) {
            (void)cudaGetLastError();
            err = std::string(what) + ": " + cudaGetErrorString(e);
            rc = ECMC_ECUDA;
        }
    };
    cu(cudaMemcpyAsync(g->d_ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, st), "ctl");
    cu(cudaMemsetAsync(g->d_bar, 0, 2 * sizeof(unsigned int), st), "bar");
    cu(cudaMemsetAsync(g->d_err, 0, sizeof(int32_t), st), "err");
    cu(cudaMemsetAsync(g->d_phase, 0, GPH_N * sizeof(unsigned long long), st), "phase");
    // member tags restart with the launch's window count
    cu(cudaMemsetAsync(g->s.memb, 0xFF, (size_t)g->s.k * 8, st), "memb");
    if (rc) return rc;
    GRun R;
    R.s = g->s;
    R.ctl = g->d_ctl;
    R.bar = g->d_bar;
    R.err = g->d_err;
    R.phase_ns = g->d_phase;
    R.max_legs = n_legs;
    R.leg0 = g->log_legs;
    R.budget = (int64_t)budget;
    void *args[] = {&R};
    cu(cudaEventRecord(g->ev0, st), "event");
    cu(cudaLaunchCooperativeKernel((void *)k_run_graph, g->grid, GRUN_THREADS, args, UF_SMEM_BYTES,
                                   st),
       "launch");
    cu(cudaEventRecord(g->ev1, st), "event");
    int32_t gerr = 0;
    unsigned long long ph[GPH_N];
    cu(cudaMemcpyAsync(&ctl, g->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost, st), "ctl");
    cu(cudaMemcpyAsync(&gerr, g->d_err, sizeof gerr, cudaMemcpyDeviceToHost, st), "err");
    cu(cudaMemcpyAsync(ph, g->d_phase, sizeof ph, cudaMemcpyDeviceToHost, st), "phase");
    cu(cudaStreamSynchronize(st), "run");
    if (rc) return rc;
    float ms = 0.f;
    cu(cudaEventElapsedTime(&ms, g->ev0, g->ev1), "elapsed");
    g->log_legs += ctl.legs;
    tot->legs = ctl.legs;
    tot->lifts = ctl.lifts;
    tot->conflict_legs = ctl.conflict_legs;
    tot->repaired = ctl.repaired;
    tot->continued = ctl.continued;
    tot->restarts = ctl.restarts;
    tot->horizon = ctl.horizon;
    tot->order_err = ctl.order_err;
    tot->p1_lifts = ctl.p1_lifts;
    tot->repair_lifts = ctl.repair_lifts;
    tot->blocked = ctl.blocked;
    tot->cwindows = ctl.cwindows;
    tot->ms = ms;
    tot->pass1_ms = ph[GPH_PASS1] * 1e-6;
    tot->repair_ms = ph[GPH_REPAIR] * 1e-6;
    tot->other_ms = (ph[GPH_BEGIN] + ph[GPH_END]) * 1e-6;
    if (legs_done) *legs_done = (int32_t)ctl.legs;
    if (flags_host && ctl.legs > 0) {
        cu(cudaMemcpy(flags_host, g->d_flags, (size_t)ctl.legs, cudaMemcpyDeviceToHost), "flags");
        if (rc) return rc;
    }
    if (gerr == ECMC_ETIMEOUT) {
        err = "a grid barrier wait passed its time limit";
        return ECMC_ETIMEOUT;
    }
    if (ctl.err) {
        err = "undo records or repair rounds overflowed";
        return ECMC_ECAPACITY;
    }
    double dg[7];
    if (cudaMemcpy(dg, g->s.dbg, sizeof dg, cudaMemcpyDeviceToHost) == cudaSuccess &&
        dg[0] != 0.0) {
        char buf[240];
        snprintf(buf, sizeof buf, "internal check %g failed: %.17g %.17g %.17g %.17g %.17g %.17g",
                 dg[0], dg[1], dg[2], dg[3], dg[4], dg[5], dg[6]);
        err = buf;
        return ECMC_ECUDA;
    }
    return 0;
}

struct GBatchScratch {
    int cap = 0;
    GDev *d_S = nullptr;
    GCtl *d_ctl = nullptr;
    int32_t *d_chain_base = nullptr, *d_comp_base = nullptr, *d_g = nullptr, *d_err = nullptr;
    unsigned int *d_bar = nullptr;
    unsigned long long *d_phase = nullptr;
    int grid = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

void graph_batch_free(GBatchScratch *b) {
    if (!b) return;
    dm_free(b->d_S);
    dm_free(b->d_ctl);
    dm_free(b->d_chain_base);
    dm_free(b->d_comp_base);
    dm_free(b->d_g);
    dm_free(b->d_err);
    dm_free(b->d_bar);
    dm_free(b->d_phase);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

int graph_batch_run(GBatchScratch **scratch, GraphCtx *const *gs, int32_t n, int32_t max_legs,
                    const uint64_t *budgets, cudaStream_t st, GraphTotals *tots,
                    int32_t *legs_out, double *ms_out, std::string &err) {
    if (ms_out) *ms_out = 0.0;
    if (n < 1 || max_legs < 0) {
        err = "bad batch size or leg count";
        return ECMC_EINVAL;
    }
    const int W = gs[0]->s.windows;
    for (int r = 0; r < n; ++r) {
        if (!gs[r] || gs[r]->s.windows != W) {
            err = "all contexts of a batch need the same claim windows";
            return ECMC_EINVAL;
        }
        if (gs[r]->s.restart) {
            err = "restart-mode contexts run alone (ecmc_run_to_breakpoint)";
            return ECMC_EINVAL;
        }
        if ((int64_t)max_legs * W >= ((int64_t)1 << 24)) {
            err = "too many legs x windows for one call (< 2^24)";
            return ECMC_EINVAL;
        }
    }
    for (int r = 0; r < n; ++r) {
        memset(&tots[r], 0, sizeof tots[r]);
        if (legs_out) legs_out[r] = 0;
    }
    if (max_legs == 0) return 0;
    GBatchScratch *b = *scratch;
    if (!b) {
        b = new (std::nothrow) GBatchScratch();
        if (!b) return ECMC_ENOMEM;
        *scratch = b;
    }
    if (b->cap < n) {
        const int cap = std::max(n, 2 * b->cap);
        dm_free(b->d_S);
        dm_free(b->d_ctl);
        dm_free(b->d_chain_base);
        dm_free(b->d_comp_base);
        b->d_S = nullptr;
        b->d_ctl = nullptr;
        b->d_chain_base = b->d_comp_base = nullptr;
        b->cap = 0;
        if (dm_alloc_t(&b->d_S, (size_t)cap * sizeof(GDev)) != 0 ||
            dm_alloc_t(&b->d_ctl, (size_t)cap * sizeof(GCtl)) != 0 ||
            dm_alloc_t(&b->d_chain_base, (size_t)(cap + 1) * 4) != 0 ||
            dm_alloc_t(&b->d_comp_base, (size_t)(cap + 1) * 4) != 0) {
            err = "batch scratch";
            return ECMC_ENOMEM;
        }
        b->cap = cap;
    }
    if (!b->d_g) {
        int dev = 0, n_sm = 1, blocks = 0;
        if (dm_alloc_t(&b->d_g, GB_N * sizeof(int32_t)) != 0 ||
            dm_alloc_t(&b->d_err, sizeof(int32_t)) != 0 ||
            dm_alloc_t(&b->d_bar, 2 * sizeof(unsigned int)) != 0 ||
            dm_alloc_t(&b->d_phase, GPH_N * sizeof(unsigned long long)) != 0 ||
            cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_run_graph_batch,
                                                          GRUN_THREADS, UF_SMEM_BYTES) !=
                cudaSuccess ||
            blocks < 1) {
            (void)cudaGetLastError();
            err = "batch scratch";
            return ECMC_ENOMEM;
        }
        b->grid = n_sm * std::min(blocks, GRUN_MIN_BLOCKS);
    }
    std::vector<GDev> S(n);
    std::vector<GCtl> ctl(n);
    std::vector<int32_t> base(n + 1, 0);
    int rc = 0;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && !rc) {
            (void)cudaGetLastError();
            err = std::string(what) + ": " + cudaGetErrorString(e);
            rc = ECMC_ECUDA;
        }
    };
    for (int r = 0; r < n; ++r) {
        GraphCtx *g = gs[r];
        if (g->st != st) cu(cudaStreamSynchronize(g->st), "context stream");
        if (g->flags_cap < max_legs) {
            dm_free(g->d_flags);
            g->d_flags = nullptr;
            g->flags_cap = 0;
            if (dm_alloc_t(&g->d_flags, (size_t)max_legs) != 0) {
                err = "flags allocation";
                return ECMC_ENOMEM;
            }
            g->flags_cap = max_legs;
        }
        S[r] = g->s;
        memset(&ctl[r], 0, sizeof(GCtl));
        ctl[r].budget = budgets ? (int64_t)budgets[r] : 0;
        ctl[r].flags = g->d_flags;
        ctl[r].flags_cap = g->flags_cap;
        ctl[r].leg0 = g->log_legs;
        base[r + 1] = base[r] + g->s.k;
        // member tags restart with the launch's window count
        cu(cudaMemsetAsync(g->s.memb, 0xFF, (size_t)g->s.k * 8, st), "memb");
    }
    if (rc) return rc;
    cu(cudaMemcpyAsync(b->d_S, S.data(), (size_t)n * sizeof(GDev), cudaMemcpyHostToDevice, st),
       "descriptors");
    cu(cudaMemcpyAsync(b->d_ctl, ctl.data(), (size_t)n * sizeof(GCtl), cudaMemcpyHostToDevice, st),
       "ctl");
    cu(cudaMemcpyAsync(b->d_chain_base, base.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice,
                       st),
       "chain base");
    cu(cudaMemsetAsync(b->d_g, 0, GB_N * sizeof(int32_t), st), "counters");
    cu(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned int), st), "bar");
    cu(cudaMemsetAsync(b->d_err, 0, sizeof(int32_t), st), "err");
    cu(cudaMemsetAsync(b->d_phase, 0, GPH_N * sizeof(unsigned long long), st), "phase");
    if (rc) return rc;
    GBatchDev B;
    B.S = b->d_S;
    B.ctl = b->d_ctl;
    B.chain_base = b->d_chain_base;
    B.comp_base = b->d_comp_base;
    B.g = b->d_g;
    B.bar = b->d_bar;
    B.err = b->d_err;
    B.phase_ns = b->d_phase;
    B.R = n;
    B.max_legs = max_legs;
    B.windows = W;
    B.pad = 0;
    void *args[] = {&B};
    cu(cudaEventRecord(b->ev0, st), "event");
    cu(cudaLaunchCooperativeKernel((void *)k_run_graph_batch, b->grid, GRUN_THREADS, args,
                                   UF_SMEM_BYTES, st),
       "launch");
    cu(cudaEventRecord(b->ev1, st), "event");
    int32_t gerr = 0;
    unsigned long long ph[GPH_N];
    cu(cudaMemcpyAsync(ctl.data(), b->d_ctl, (size_t)n * sizeof(GCtl), cudaMemcpyDeviceToHost, st),
       "ctl");
    cu(cudaMemcpyAsync(&gerr, b->d_err, sizeof gerr, cudaMemcpyDeviceToHost, st), "err");
    cu(cudaMemcpyAsync(ph, b->d_phase, sizeof ph, cudaMemcpyDeviceToHost, st), "phase");
    cu(cudaStreamSynchronize(st), "run");
    if (rc) return rc;
    float ms = 0.f;
    cu(cudaEventElapsedTime(&ms, b->ev0, b->ev1), "elapsed");
    if (ms_out) *ms_out = ms;
    bool cap_err = false;
    for (int r = 0; r < n; ++r) {
        const GCtl &c = ctl[r];
        gs[r]->log_legs += c.legs;
        GraphTotals &t = tots[r];
        t.legs = c.legs;
        t.lifts = c.lifts;
        t.conflict_legs = c.conflict_legs;
        t.repaired = c.repaired;
        t.continued = c.continued;
        t.horizon = c.horizon;
        t.order_err = c.order_err;
        t.p1_lifts = c.p1_lifts;
        t.repair_lifts = c.repair_lifts;
        t.blocked = c.blocked;
        t.cwindows = c.cwindows;
        if (n == 1) {
            t.ms = ms;
            t.pass1_ms = ph[GPH_PASS1] * 1e-6;
            t.repair_ms = ph[GPH_REPAIR] * 1e-6;
            t.other_ms = (ph[GPH_BEGIN] + ph[GPH_END]) * 1e-6;
        }
        if (legs_out) legs_out[r] = (int32_t)c.legs;
        if (c.err) cap_err = true;
    }
    if (gerr == ECMC_ETIMEOUT) {
        err = "a grid barrier wait passed its time limit";
        return ECMC_ETIMEOUT;
    }
    if (cap_err) {
        err = "undo records or repair rounds overflowed";
        return ECMC_ECAPACITY;
    }
    return 0;
}

int graph_export(GraphCtx *g, double *x, double *y, double *t, int32_t *active) {
    const GDev &s = g->s;
    cudaStream_t st = g->st;
    if (x || t) k_g_export<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s, x, t);
    if (y) cudaMemcpyAsync(y, s.y, (size_t)s.n * 8, cudaMemcpyDeviceToDevice, st);
    if (active) k_g_export_active<<<(unsigned)((s.k + 127) / 128), 128, 0, st>>>(s, active);
    return cudaGetLastError() == cudaSuccess ? 0 : ECMC_ECUDA;
}

int graph_arrows(GraphCtx *g, int32_t *a, double *b, std::string &err) {
    const GDev &s = g->s;
    cudaStream_t st = g->st;
    // strided copies straight out of the 64-byte records
    cudaError_t e = cudaSuccess;
    if (a)
        e = cudaMemcpy2DAsync(a, 3 * sizeof(uint32_t), &s.g[0].a[0], sizeof(GDisk),
                              3 * sizeof(uint32_t), (size_t)s.n, cudaMemcpyDeviceToHost, st);
    if (b && e == cudaSuccess)
        e = cudaMemcpy2DAsync(b, 3 * sizeof(double), &s.g[0].b[0], sizeof(GDisk),
                              3 * sizeof(double), (size_t)s.n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        err = std::string("graph arrows: ") + cudaGetErrorString(e);
        return ECMC_ECUDA;
    }
    return 0;
}

int graph_transpose(GraphCtx *g, std::string &err) {
    GDev &s = g->s;
    double *xnew = nullptr;
    if (dm_alloc_t(&xnew, (size_t)s.n * 8) != 0) {
        err = "transpose scratch";
        return ECMC_ENOMEM;
    }
    k_g_swap_xy<<<(unsigned)((s.n + 255) / 256), 256, 0, g->st>>>(s, xnew);
    k_g_reset_chains<<<(unsigned)((s.k + 127) / 128), 128, 0, g->st>>>(s);
    int rc = graph_build(g, xnew, s.y, err);  // x, t = 0 and arrows for the new frame
    // (the build's kernels read xnew: done before the block goes back)
    if (cudaStreamSynchronize(g->st) != cudaSuccess && rc == 0) {
        (void)cudaGetLastError();
        err = "transpose";
        rc = ECMC_ECUDA;
    }
    dm_free(xnew);
    return rc;
}

int graph_liftings(GraphCtx *g, ecmc_lift_t *buf, int64_t cap, int64_t *n_out,
                   std::string &err) {
    const GDev &s = g->s;
    if (!s.log_on) {
        err = "lifting log not enabled";
        return ECMC_EINVAL;
    }
    unsigned long long n = 0;
    if (cudaMemcpy(&n, s.tc_cnt + TC_LOG_N, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        err = "log count";
        return ECMC_ECUDA;
    }
    *n_out = (int64_t)n;
    if ((int64_t)n > s.log_cap) {
        err = "lifting log overflowed log_cap";
        return ECMC_ECAPACITY;
    }
    std::vector<ecmc_lift_t> all((size_t)n);
    if (n && cudaMemcpy(all.data(), s.log, n * sizeof(ecmc_lift_t), cudaMemcpyDeviceToHost) !=
                 cudaSuccess) {
        err = "log copy";
        return ECMC_ECUDA;
    }
    std::stable_sort(all.begin(), all.end(), [](const ecmc_lift_t &a, const ecmc_lift_t &b) {
        return a.leg != b.leg ? a.leg < b.leg : a.c < b.c;
    });
    if (buf && cap > 0)
        memcpy(buf, all.data(), (size_t)std::min<int64_t>(cap, (int64_t)n) * sizeof(ecmc_lift_t));
    return 0;
}

void graph_destroy(GraphCtx *g) {
    if (!g) return;
    if (cudaStreamSynchronize(g->st) != cudaSuccess) (void)cudaGetLastError();
    for (void *p : g->allocs) dm_free(p);
    for (void *p : g->build_tmp) dm_free(p);
    dm_free(g->d_flags);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

int64_t graph_device_bytes(const GraphCtx *g) { return g ? g->bytes : 0; }

int64_t graph_plan_bytes(const ecmc_params *p, int nc) {
    GraphCtx *g = new (std::nothrow) GraphCtx();
    if (!g) return -1;
    GDev &s = g->s;
    memset(&s, 0, sizeof s);
    s.cap = p->undo_cap > 0 ? p->undo_cap : 1024;
    s.log_on = (p->flags & ECMC_LOG_LIFTINGS) ? 1 : 0;
    s.log_cap = s.log_on ? (p->log_cap > 0 ? p->log_cap : ((int64_t)1 << 22)) : 0;
    std::string err;
    int64_t total = -1;
    if (graph_plan(g, p, err) == 0) {
        total = 0;
        for (auto &r : g->pending) total += (int64_t)((r.second + 255) & ~(size_t)255);
        const double a = p->box / nc;
        const int C = a < std::sqrt(2.0) * p->d * (1.0 - 1e-9) ? 4 : 8;
        total += graph_build_bytes(p->box, p->d, nc, C);
    }
    g->pending.clear();
    delete g;
    return total;
}
