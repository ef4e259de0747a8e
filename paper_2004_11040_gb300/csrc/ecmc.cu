// ecmc.cu -- libecmc: multithreaded event-chain Monte Carlo for hard disks on
// one GPU (sm_103a), after Li, Todo, Maggs & Krauth, "Multithreaded event-chain
// Monte Carlo with local times" (arXiv:2004.11040).
//
// Design (one leg = one interval [h, h'] between breakpoints, v = (1, 0)):
//   * Disks live in square cells of side a = L/nc > d, stored as per-slot
//     structure-of-arrays (x, y, id); C slots per cell (C = 4 for a < sqrt(2) d).
//   * One warp runs one chain (one task of Alg. 5/6): lanes cover
//     3 rows x C slots of one or two columns ahead of the active disk, compute
//     the time of flight tau_j = dx_j - sqrt(d^2 - dy_j^2) in FP64 (Sec. 2.2),
//     and reduce (tau, j) with warp shuffles.
//   * Before a chain may use a cell it claims it for the leg with atomicCAS on
//     a per-cell word (Alg. 5's compare-and-swap, lifted from disks to cells). Cells
//     therefore change only under their claimer, and a chain that meets a cell
//     claimed by another chain stops: the leg's conflict flag. A cell whose
//     row holds no disk within d in y of the active disk (y never changes
//     along x) is claimed weakly and not read: it counts for the flag but
//     blocks nobody. The target disk is also claimed with atomicCAS on its
//     per-disk owner word (Alg. 5's compare-and-swap on the target's tag).
//   * Without a conflict every chain followed exactly the path it would take
//     alone, which equals the global-time result (Lemma 2). With a conflict
//     the chains that met (connected components of the conflict graph) are
//     rolled back to the earliest time T* at which one of them was blocked --
//     their events before T* are exact -- and one warp per component redoes
//     them from T* in global event-time order (Alg. 2). A component that meets
//     a cell of another chain stops and merges with it in the next round.
//     This is the first restart strategy of Sec. 3.4, made exact and local.
// All FP64 arithmetic uses explicit round-to-nearest intrinsics (and the file
// is compiled with -fmad=false) so that results are reproducible bit for bit.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "devmem.h"
#include "ecmc.h"
#include "graph.h"

namespace {

constexpr uint32_t REC_NO_OWNER = 1u;  // the target's owner word was not taken

// One event of a chain: enough to undo it exactly, and the lifting (Eq. 1).
struct Rec {
    uint32_t i, from, to, j;  // moved disk, its slot before/after, target (NONE: stall)
    uint32_t jloc, seq;       // slot of j; order of application within its run
    uint32_t flags, pad;
    double x_old;             // x of i before the move
    double ti_old, tj_old;    // local times of i and j before the event
    double t, tau, xi, xj;    // event time (= new t_j), time of flight, x_i at contact, x_j
    double d_after;           // remaining chain length after the event
};

struct Dev {
    int64_t n;
    int nc, k, cap, windows;
    double L, d, d2, ell, a, inv_a, eps;
    double far;  // L - 3a: a chain with less than this left never lifts onto a
                 // disk behind its active disk (that is more than L - 2a ahead)
    // Exact tables of the cell map (null: computed in FP64):
    const double *colx;                // [nc] RN(c a), the left edge of column c
    const unsigned long long *xbound;  // [nc + 1] least x (bits) with
                                       // cell_coord(x) >= c; [0] = 0, [nc] = +inf
    // FP32 image of the scan's stop rule: |thr_f - lim_f - (thr - lim)| <= stop_e / 2
    float af, df, epsf, stop_e;
    // cells: slot q of cell c at index c*C + q; a disk's x, y, local time and
    // owner word live in its slot and move with it
    double *cx, *cy, *ct;
    uint32_t *cid, *cown;
    // rows a disk's scan need not read (moves along x never change a disk's
    // cell row): bit 0 the row below, bit 1 the row above, when no disk of
    // that row lies within d in y; per slot, moving with the disk (or null:
    // every row is read)
    uint8_t *cskp;
    unsigned long long *rband;  // [2 nc]: least and largest y (bits) per cell row
    // per cell: 0, chain+1 (the chain reads the cell) or chain+1 | CLAIM_WEAK
    // (the chain's scan covers the cell but need not read it)
    uint32_t *claim;
    // per chain
    uint32_t *aloc0, *aloc;
    uint32_t *ci;  // active disk id
    double *D, *tc;
    int32_t *status, *partner, *nrec, *nlift;
    Rec *rec;  // [k * cap]
    // pending events for the global-time repair of large components
    double *ev_T, *ev_tau, *ev_xj, *ev_yj, *ev_tj;
    uint32_t *ev_j, *ev_jloc;
    int32_t *ev_lift, *ev_cx, *ev_cy, *ev_mlast;
    // conflict components
    double *vt;          // per chain: its events are exact before this time
    int32_t *uf;         // union-find parent
    int32_t *fin;        // 0: in a component to repair; 1: final since the round began;
                         // 2: made final in this round (by its component's repair)
    int32_t *comp_of;    // component root per chain
    int32_t *abort_to;   // chain met by an aborted component (per root), -1
    int32_t *comp_cnt;   // members per root (dirty components)
    int32_t *comp_off;   // [k+1] offsets of dirty components
    int32_t *comp_root;  // root of the q-th dirty component
    int32_t *comp_mem;   // members, grouped by component
    int32_t *blist;      // [k] the window's blocked chains (their count: LC_WBLOCKED)
    int32_t *pcnt;       // [k] blocked chains naming the chain as partner (0 between uses)
    int32_t *ctl;        // [CTL_N]
    unsigned long long *lc;      // [LC_N]
    unsigned long long *tc_cnt;  // [TC_N]
    ecmc_lift_t *log;
    int64_t log_cap;
    int log_on;
    double *dbg;  // [16] first failed internal check (diagnostics)
    // row pass (rowpass.cuh): claim keys, least and largest claiming chain per
    // cell; per-system counters by window parity; the end of each chain's
    // speculative run
    int rp_ok;                   // the context may use the row pass
    unsigned long long *ckey;    // [ncell], ~0 when unclaimed
    uint32_t *camin, *camax;     // [ncell], chain + 1; ~0 and 0 when unclaimed
    int32_t *rp;                 // [RP_N]: chains not eligible (by window parity), cancels
    int32_t *rp_n, *rp_front, *rp_end, *rp_partner;
    uint32_t *rp_aloc, *rp_ci, *rp_start;
    double *rp_tc, *rp_D;
};

// Record e of chain c. Records are stored by event index, then chain: the
// first events of a leg of all chains lie in one dense block (one page per
// chain, as with chain-major storage, costs a translation miss per chain).
__device__ __forceinline__ Rec *rec_at(const Dev &s, int c, int e) {
    return s.rec + (size_t)e * (size_t)s.k + (size_t)c;
}

// ------------------------------------------------------------ FP64 geometry

// Records the first failed internal check: kind, then up to 6 values.
__device__ void diag(const Dev &s, int kind, double a, double b, double c, double d, double e,
                     double f) {
    if (!s.dbg) return;
    if (atomicCAS((unsigned long long *)s.dbg, 0ull, (unsigned long long)__double_as_longlong((double)kind)) != 0ull)
        return;
    s.dbg[1] = a;
    s.dbg[2] = b;
    s.dbg[3] = c;
    s.dbg[4] = d;
    s.dbg[5] = e;
    s.dbg[6] = f;
}

__device__ __forceinline__ int cell_coord(double v, const Dev &s) {
    int c = __double2int_rz(__dmul_rn(v, s.inv_a));
    if (c >= s.nc) c = s.nc - 1;
    if (c < 0) c = 0;
    return c;
}

__device__ __forceinline__ uint32_t cell_of(double x, double y, const Dev &s) {
    return (uint32_t)cell_coord(y, s) * (uint32_t)s.nc + (uint32_t)cell_coord(x, s);
}

// v rounded toward zero to FP32 on the integer pipe (a conversion on this
// chip's FP64 pipe would occupy it ~64 cycles per warp instruction, whatever
// the lane mask, with ~60 cycles of dependent latency): relative error below
// 2^-23, and
// |v| < 2^-126 gives 0.
__device__ __forceinline__ float d2f_trunc(double v) {
    const unsigned long long b = dbits(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FFull) - 1023;
    if (e < -126) return __int_as_float((int)sign);
    if (e > 127) return __int_as_float((int)(sign | 0x7F800000u));
    return __int_as_float(
        (int)(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFull)));
}

// The stop rule in FP64 as defined (a call of its own, so that the compiler
// never evaluates its five FP64 instructions -- ~64 cycles of the FP64 unit
// each on this GPU -- on the path where the FP32 image decides).
__device__ __noinline__ bool beyond_exact(double a, double d, double eps, int m, double fx,
                                          unsigned long long cur) {
    const double thr = __dsub_rn(__dsub_rn(__dmul_rn((double)m, a), fx), d);
    const double lim = __dadd_rn(__longlong_as_double((long long)cur), eps);
    return !dneg(thr) && dbits(thr) > dbits(lim);
}

// The constants of the stop rule, held in registers by the callers' loops.
struct StopK {
    float af, df, epsf, stop_e;
    double a, d, eps;
};

__device__ __forceinline__ StopK stopk_of(const Dev &s) {
    StopK k;
    k.af = s.af;
    k.df = s.df;
    k.epsf = s.epsf;
    k.stop_e = s.stop_e;
    k.a = s.a;
    k.d = s.d;
    k.eps = s.eps;
    return k;
}

// The scan's stop rule: is thr(m) = ((m a) - fx) - d above RN(cur + eps)?
// Decided on the FP32 image thr_f - lim_f when that lies farther than stop_e
// from 0 (its error bound is stop_e / 4, so the answer is the exact one),
// else in FP64 as defined. lim_f = trunc(cur) + eps in FP32.
__device__ __forceinline__ bool beyond_k(const StopK &k, int m, double fx, float fxf, float lim_f,
                                         unsigned long long cur) {
    if (k.stop_e > 0.f) {
        const float thr_f = __fsub_rn(__fsub_rn(__fmul_rn(__int2float_rn(m), k.af), fxf), k.df);
        const float diff = __fsub_rn(thr_f, lim_f);
        if (diff > k.stop_e) return true;
        if (diff < -k.stop_e) return false;
    }
    return beyond_exact(k.a, k.d, k.eps, m, fx, cur);
}

__device__ __forceinline__ bool beyond(const Dev &s, int m, double fx, float fxf, float lim_f,
                                       unsigned long long cur) {
    return beyond_k(stopk_of(s), m, fx, fxf, lim_f, cur);
}

// thr(m) <= eps, where a column is scanned (and its cells claimed) whatever
// the candidates: true only where certain (m = 0, or the FP32 image is below
// eps by more than its error bound); false answers only delay claims.
__device__ __forceinline__ bool surely_scanned(const Dev &s, int m, float fxf) {
    if (m == 0) return true;
    if (!(s.stop_e > 0.f)) return false;
    const float thr_f = __fsub_rn(__fsub_rn(__fmul_rn(__int2float_rn(m), s.af), fxf), s.df);
    return thr_f < __fsub_rn(s.epsf, s.stop_e);
}

// cell_of(x, y) of a disk that moved along x out of cell cell_old: the row
// is unchanged, and the column is the last c with xbound[c] <= x (integer
// compares of non-negative doubles), searched from the old column, or from 0
// once x wrapped around the box. Long moves, or no table: cell_of.
__device__ __forceinline__ uint32_t cell_after_move(const Dev &s, uint32_t cell_old, double x,
                                                    double y) {
    if (s.xbound) {
        const uint32_t nc = (uint32_t)s.nc, row = cell_old / nc;
        uint32_t col = cell_old % nc;
        const unsigned long long xb = dbits(x);
        if (xb < s.xbound[col]) col = 0;
        for (int it = 0; it < 4; ++it) {
            if (col + 1 >= nc || xb < s.xbound[col + 1]) return row * nc + col;
            ++col;
        }
    }
    return cell_of(x, y, s);
}

__device__ __forceinline__ double wrap_add(double x, double dx, const Dev &s) {
    double r = __dadd_rn(x, dx);
    if (dbits(r) >= dbits(s.L)) r = __dsub_rn(r, s.L);  // r >= 0
    return r;
}


// ------------------------------------------------------------- one step

enum { MODE_PASS1 = 0, MODE_COMP = 1, MODE_CONT = 2 };

struct ChainReg {
    uint32_t i, iloc;
    double xi, yi, ti, D;
    uint32_t skip;  // rows of the footprint the scan need not read (cskp)
};

constexpr uint32_t CLAIM_WEAK = 0x80000000u;

__device__ __forceinline__ uint32_t skip_of(const Dev &s, uint32_t loc) {
    return s.cskp ? (uint32_t)s.cskp[loc] : 0u;
}

struct StepOut {
    double tau;  // tau* (lift) or D (stall)
    uint32_t j, jloc;
    double xj, yj, tj;
    int lift;
    int cx, cy, mlast;  // scanned footprint: rows cy-1..cy+1, columns cx..cx+mlast
    int conflict;
    uint32_t partner;
    // a run of Alg. 4 stops here (Remark 10, taken conservatively): another
    // chain's active or stalled disk in a scanned corridor lies within reach
    // (its time of flight is below D) or fails Eq. 2; ns_owner is the chain of
    // the nearest one
    int nonstatic;
    uint32_t ns_owner;
    int viol;       // CONT: a scanned corridor disk fails the horizon condition (Eq. 2)
    // PASS1: the scan met another chain's claim on a cell it need not read, or
    // took over another chain's weak claim: the claim sets overlap (the flag)
    int weak;
    uint32_t jskp;  // skip bits of the target's slot
    // empty slots of the middle row (the active disk's row) as scanned: C bits
    // per column offset m (bit m*C + slot), for the columns with (m+1)*C <= 64
    unsigned long long emask;
};

// The next event of one chain (time of flight to every candidate and the
// least (tau, j), Sec. 2.2), with the cell scan: columns ahead
// of the active disk are scanned until (m*a - fx) - d > min(D, best) + eps.
// Every scanned cell is claimed for the leg (conflict if another owner holds
// it strongly; weakly, without a read, where the row is out of reach in y).
// A column whose threshold is <= eps is scanned whatever the candidates, so
// its cells are claimed together with their load.
// In both modes the active and stalled disks of all chains are excluded
// (Alg. 2), and a static disk with t_i + tau < t_j became static after the
// chain's disk had passed it (lazy per-chain frame): it is one lap away.
// Reading the owner word in pass 1 as well keeps every pass-1 event of a
// claim window at or after the window start: a lift onto another chain's
// active disk could otherwise land before it (zero flight time from contact).
// PASS1: the owner is the chain. A disk with t_i + tau < t_j whose t_j lies in
//   the current window (start tw) would be a horizon violation (Eq. 2); it
//   cannot occur while the cells are held and is counted as an assertion.
// COMP: the owner is the conflict component `root` (any member's claim is its
//   own).
// CONT: as COMP, and the scan runs until (m*a - fx) - d > D + eps: the
//   horizon condition must hold for the nearest disk of every corridor within
//   reach (Lemma 2; the arrows of G(3)), not only for those before the winner.
//   A disk another member moved can sit beyond the winner in one corridor
//   while the continued chain's earlier sweep crossed its old place.
__device__ void uf_union(int32_t *p, int a, int b);

// nm > 0 (COMP, CONT): the component's members are the chains my_member of
// lanes 0..nm-1, so a claim's holder is tested with shuffles instead of a
// load; nm = 0: by comp_of; nm < 0 (CONT): the -nm members in the lanes'
// registers, then comp_of, and a chain that is in no component is taken
// over by this one.
template <int C, int MODE>
__device__ StepOut scan_step(const Dev &s, int c, int root, const ChainReg &r, double tw,
                             int nm = 0, int my_member = -1) {
    constexpr int LPC = (3 * C <= 16) ? 16 : 32;  // lanes per column
    constexpr int CPP = 32 / LPC;                 // columns per pass
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPC, sub = lane % LPC;
    const int rr = sub / C, sl = sub % C;
    const bool used = sub < 3 * C;
    const int nc = s.nc;
    const uint32_t mine = (uint32_t)c + 1u;
    const uint32_t mine_w = mine | CLAIM_WEAK;
    // a row none of whose disks lies within d in y of the active disk holds no
    // candidate: its slots are not read, and in pass 1 its cells are claimed
    // weakly (the claim set, hence the flag, is that of the full scan)
    const bool need = rr == 1 || !((r.skip >> (rr >> 1)) & 1u);

    // the active disk's cell is that of its slot (cells always hold the
    // disks whose coordinates fall in them)
    const int cxi = (int)((r.iloc / C) % (uint32_t)nc), cyi = (int)((r.iloc / C) / (uint32_t)nc);
    const double fx = __dsub_rn(r.xi, s.colx ? s.colx[cxi] : __dmul_rn((double)cxi, s.a));
    const float fxf = d2f_trunc(fx);
    int row = cyi + rr - 1;
    if (row < 0) row += nc;
    if (row >= nc) row -= nc;

    // warp-uniform skips of arithmetic no lane needs (results unchanged): the
    // periodic minimum in y only where the scanned rows wrap around the box
    // (elsewhere |dy| < 2a < L/2), and a disk behind the active disk in its
    // own column (more than L - 2a ahead) only when D could reach it
    const bool ywrap = cyi == 0 || cyi == nc - 1 || nc <= 4;
    const bool near_d = !(dbits(r.D) < dbits(s.far));
    unsigned long long cur = dbits(r.D);  // min(D, best tau so far): drives the stop rule
    float lim_f = __fadd_rn(d2f_trunc(r.D), s.epsf);  // its FP32 image, + eps
    unsigned long long btau = INF_BITS;
    double bx = 0.0, by = 0.0, bt = 0.0;
    uint32_t bj = NONE, bloc = 0, bskp = 0;
    int mlast = 0;
    bool stop = false;
    bool conflict = false;
    uint32_t partner = NONE;
    bool hz = false;
    unsigned long long ns_t = INF_BITS;  // least time of flight to another chain's disk
    uint32_t ns_own = NONE;                // ... and its chain
    bool ns_hv = false;                    // such a disk fails Eq. 2 (this lane)
    bool viol = false;   // CONT: a scanned corridor disk fails Eq. 2
    bool weakc = false;  // PASS1: claim sets overlap on a weak claim (this lane)
    unsigned long long emask = 0ull;

    for (int m0 = 0; m0 < nc && !stop; m0 += CPP) {
        const int m = m0 + grp;
        const bool colok = used && m < nc;
        int col = cxi + m;
        if (col >= nc) col -= nc;
        const uint32_t cell = (uint32_t)row * (uint32_t)nc + (uint32_t)col;
        const uint32_t loc = cell * C + sl;
        // a column whose threshold is <= eps is scanned in any case
        const bool certain = surely_scanned(s, m, fxf);
        // all loads of the slot at once (an empty slot's values are ignored;
        // they share the cell's sectors with the occupied ones). They are
        // issued before the claim so that both round trips overlap: a cell
        // read before its claim succeeds was not written in this window
        // (claims are taken before writes and never released in a window),
        // and a failed claim discards what was read.
        uint32_t id = EMPTY, own = OWN_STATIC, skp = 0;
        double xj = 0.0, yj = 0.0, tj = 0.0;
        // claim word: the raw result of the CAS (claimed_early) or the value
        // read; turned into the holder only where the conflict test needs it
        uint32_t claim_w = 0;
        bool claimed_early = false;
        const uint32_t word = need ? mine : mine_w;
        if (colok && need) {
            id = s.cid[loc];
            xj = s.cx[loc];
            yj = s.cy[loc];
            tj = s.ct[loc];
            own = s.cown[loc];
            if (s.cskp) skp = s.cskp[loc];
        }
        // repairs claim only the cells they read
        if (colok && sl == 0 && (need || MODE == MODE_PASS1)) {
            if (certain) {
                claim_w = atomicCAS(s.claim + cell, 0u, word);
                claimed_early = true;
            } else {
                // through L2: claims are reset between windows by other SMs, so
                // an L1 line from an earlier window could still show this
                // chain's claim
                claim_w = __ldcg(s.claim + cell);
            }
        }
        const bool cand = id != EMPTY && id != r.i;
        {
            const unsigned eb = __ballot_sync(FULL, colok && rr == 1 && id == EMPTY);
#pragma unroll
            for (int g = 0; g < CPP; ++g) {
                const int mc = m0 + g;
                if ((mc + 1) * C <= 64)
                    emask |= (unsigned long long)((eb >> (g * LPC + C)) & ((1u << C) - 1u))
                             << (mc * C);
            }
        }
        // time of flight of i towards j (Sec. 2.2: tau = x_j - x_i
        // - b_ij with b_ij = sqrt(d^2 - dy^2)): forward image in x, minimum
        // image in y, corridor |dy| < d, +inf outside, clamped at 0
        const bool cst = cand && own == OWN_STATIC;
        double ay = fabs(__dsub_rn(yj, r.yi));
        if (ywrap) {
            const double la = __dsub_rn(s.L, ay);
            if (dbits(la) < dbits(ay)) ay = la;
        }
        const bool corr = cst && dbits(ay) < dbits(s.d);
        const bool ncs = cand && own != OWN_STATIC && dbits(ay) < dbits(s.d);
        double b = 0.0;
        if (__any_sync(FULL, corr || ncs)) b = __dsqrt_rn(__dsub_rn(s.d2, __dmul_rn(ay, ay)));
        double dx = __dsub_rn(xj, r.xi);
        const bool neg = dneg(dx);
        const bool drop = neg && m == 0 && !near_d;
        const bool needl = corr && neg && !drop;
        if (__any_sync(FULL, needl) && needl) dx = __dadd_rn(dx, s.L);
        double tau = INFINITY;
        if (corr && !drop) {
            tau = __dsub_rn(dx, b);
            if (dneg(tau)) tau = 0.0;
        }
        // lazy frame: a disk that became static after the active disk passed
        // it (t_i + tau < t_j) is one lap away; t_j = +0 never is
        bool behind = false, hzv = false;
        const bool tnz = tau != INFINITY && dbits(tj) != 0ull;
        if (__any_sync(FULL, tnz)) {
            const double sum = __dadd_rn(r.ti, tau);
            behind = tnz && dbits(sum) < dbits(tj);
            // the horizon condition t_i + tau_ij > t_j (Eq. 2, strict)
            if (MODE == MODE_CONT) hzv = tnz && !(dbits(sum) > dbits(tj));
            if (__any_sync(FULL, behind) && behind) tau = __dadd_rn(tau, s.L);
        }
        const unsigned long long tb = dbits(tau);
        // (tau, j) minimum of each column (an aligned group of LPC lanes), then
        // of the pass's other column: every lane ends with both
        unsigned long long g0t = tb;
        uint32_t g0j = tb != INF_BITS ? id : NONE, g0l = loc;
#pragma unroll
        for (int o = 1; o < LPC; o <<= 1) {
            const unsigned long long t2 = shfl_xor_u64(g0t, o);
            const uint32_t j2 = __shfl_xor_sync(FULL, g0j, o);
            const uint32_t l2 = __shfl_xor_sync(FULL, g0l, o);
            if (t2 < g0t || (t2 == g0t && j2 < g0j)) {
                g0t = t2;
                g0j = j2;
                g0l = l2;
            }
        }
        unsigned long long g1t = INF_BITS;
        uint32_t g1j = NONE, g1l = 0;
        if (CPP == 2) {
            const unsigned long long t2 = shfl_xor_u64(g0t, LPC);
            const uint32_t j2 = __shfl_xor_sync(FULL, g0j, LPC);
            const uint32_t l2 = __shfl_xor_sync(FULL, g0l, LPC);
            if (grp == 0) {
                g1t = t2;
                g1j = j2;
                g1l = l2;
            } else {
                g1t = g0t;
                g1j = g0j;
                g1l = g0l;
                g0t = t2;
                g0j = j2;
                g0l = l2;
            }
        }
        // stop rule, uniform: column m0 is scanned (m0 = 0, or the previous
        // pass found its threshold within reach); the second column if its
        // threshold is within min(D, best) + eps
        int last_here = m0;
        mlast = m0;
        bool improved = false;
        if (g0t < btau || (g0t == btau && g0j < bj)) {
            btau = g0t;
            bj = g0j;
            bloc = g0l;
            improved = true;
        }
        // (a continued step checks Eq. 2 on every corridor disk within reach
        // of D, so its scan does not stop at the best candidate)
        if (MODE != MODE_CONT && g0t < cur) {
            cur = g0t;
            lim_f = __fadd_rn(d2f_trunc(__longlong_as_double((long long)cur)), s.epsf);
        }
        if (CPP == 2) {
            if (m0 + 1 >= nc || beyond(s, m0 + 1, fx, fxf, lim_f, cur)) {
                stop = true;
            } else {
                last_here = m0 + 1;
                mlast = m0 + 1;
                if (g1t < btau || (g1t == btau && g1j < bj)) {
                    btau = g1t;
                    bj = g1j;
                    bloc = g1l;
                    improved = true;
                }
                if (MODE != MODE_CONT && g1t < cur) {
                    cur = g1t;
                    lim_f = __fadd_rn(d2f_trunc(__longlong_as_double((long long)cur)), s.epsf);
                }
            }
        }
        const bool scanned = colok && m <= last_here;
        if (improved) {
            const unsigned own_lane = __ballot_sync(FULL, scanned && id == bj && loc == bloc);
            const int src = own_lane ? __ffs(own_lane) - 1 : 0;
            bx = __shfl_sync(FULL, xj, src);
            by = __shfl_sync(FULL, yj, src);
            bt = __shfl_sync(FULL, tj, src);
            bskp = __shfl_sync(FULL, skp, src);
        }
        uint32_t holder = claimed_early ? (claim_w == 0u ? word : claim_w) : claim_w;
        // lanes that hold a cell's claim word
        const bool cl = scanned && sl == 0 && (need || MODE == MODE_PASS1);
        if (cl && !claimed_early && holder == 0u) {
            const uint32_t old = atomicCAS(s.claim + cell, 0u, word);
            holder = old == 0u ? word : old;
        }
        // A cell the step reads takes over a weak claim, its own or another
        // chain's (whose holder neither read nor wrote the cell; another
        // chain's means the claim sets overlap). A weak claim only ever turns
        // into a strong one, so a failed exchange leaves a strong holder.
        if (cl && need && (holder & CLAIM_WEAK)) {
            if (MODE == MODE_PASS1 && holder != mine_w) weakc = true;
            const uint32_t old = atomicCAS(s.claim + cell, holder, mine);
            holder = old == holder ? mine : old;
        }
        bool foreign = false;
        if (MODE == MODE_PASS1) {
            if (cl && !need) {
                // a cell the step need not read never blocks it
                if (holder != mine && holder != mine_w) weakc = true;
            } else {
                foreign = cl && holder != mine;
            }
        } else if (nm != 0) {
            const int hq = cl ? (int)(holder - 1u) : -1;
            bool member = hq < 0;
            const int nmem = nm > 0 ? nm : -nm;
            for (int q = 0; q < nmem; ++q) member |= __shfl_sync(FULL, my_member, q) == hq;
            if (MODE == MODE_CONT && nm < 0 && !member) {
                // not a listed member: taken over earlier, or takeable now
                const int h = hq;
                int hc = __ldcg(s.comp_of + h);
                if (hc == h && hc != root && __ldcg(s.fin + h) == 1) {
                    const int old = atomicCAS(s.comp_of + h, h, root);
                    if (old == h) {
                        // its cells now hold this component's events: a later
                        // merge that reaches it must take the component along
                        uf_union(s.uf, h, root);
                        hc = root;
                    } else if (old == root) {
                        hc = root;
                    }
                }
                member = hc == root;
            }
            foreign = !member;
        } else if (cl) {
            foreign = __ldcg(s.comp_of + (holder - 1u)) != root;
        }
        if (foreign) {
            conflict = true;
            partner = holder - 1u;
        }
        // Eq. 2 on every scanned candidate touched in this window:
        // cannot fail while the cells are held by a lone chain; an assertion.
        if (MODE == MODE_PASS1 && scanned && behind && dbits(tj) >= dbits(tw)) hz = true;
        // another chain's active or stalled disk in a scanned corridor: its
        // time of flight (forward image, clamped) and Eq. 2
        const bool nsl = scanned && ncs;
        if (__any_sync(FULL, nsl)) {
            unsigned long long nt = INF_BITS;
            uint32_t no = NONE;
            if (nsl) {
                double dn = __dsub_rn(xj, r.xi);
                if (dneg(dn)) dn = __dadd_rn(dn, s.L);
                double tn = __dsub_rn(dn, b);
                if (dneg(tn)) tn = 0.0;
                nt = dbits(tn);
                no = own & OWN_CHAIN;
                if (dbits(tj) != 0ull && !(dbits(__dadd_rn(r.ti, tn)) > dbits(tj))) ns_hv = true;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t2 = shfl_xor_u64(nt, o);
                const uint32_t o2 = __shfl_xor_sync(FULL, no, o);
                if (t2 < nt || (t2 == nt && o2 < no)) {
                    nt = t2;
                    no = o2;
                }
            }
            if (nt < ns_t) {
                ns_t = nt;
                ns_own = no;
            }
        }
        if (MODE == MODE_CONT && scanned && hzv) viol = true;
        if (beyond(s, m0 + CPP, fx, fxf, lim_f, cur)) break;
    }

    StepOut o;
    o.cx = cxi;
    o.cy = cyi;
    o.mlast = mlast;
    o.emask = emask;
    o.nonstatic = (__ballot_sync(FULL, ns_hv) != 0u) || ns_t < dbits(r.D);
    o.ns_owner = ns_own;
    o.viol = MODE == MODE_CONT ? __ballot_sync(FULL, viol) != 0u : 0;
    o.weak = MODE == MODE_PASS1 ? __ballot_sync(FULL, weakc) != 0u : 0;
    o.conflict = 0;
    o.partner = NONE;
    const unsigned cb = __ballot_sync(FULL, conflict);
    if (cb) {
        o.conflict = 1;
        o.partner = __shfl_sync(FULL, partner, __ffs(cb) - 1);
    }
    if (MODE == MODE_PASS1 && !cb) {
        // only a step whose cells are all held is checked: a conflicting one
        // may have read a cell while its holder wrote it, and is discarded
        const unsigned hb = __ballot_sync(FULL, hz);
        if (hb && lane == __ffs(hb) - 1) atomicAdd(s.lc + LC_HORIZON, 1ull);
    }
    if (btau < dbits(r.D)) {
        o.lift = 1;
        o.tau = __longlong_as_double((long long)btau);
        o.j = bj;
        o.jloc = bloc;
        o.xj = bx;
        o.yj = by;
        o.tj = bt;
        o.jskp = bskp;
    } else {
        o.lift = 0;
        o.tau = r.D;
        o.j = NONE;
        o.jloc = 0;
        o.xj = 0.0;
        o.yj = 0.0;
        o.tj = 0.0;
        o.jskp = 0;
    }
    return o;
}

// Moves the active disk (by tau to contact, or by D to the breakpoint) with
// its local time and owner word; returns its new slot or EMPTY on a full cell.
template <int C>
__device__ uint32_t move_active(const Dev &s, const ChainReg &r, const StepOut &o, double xnew,
                                double tnew, uint32_t own_new) {
    const int lane = threadIdx.x & 31;
    const uint32_t cell_old = r.iloc / C;
    const uint32_t cell_new = cell_after_move(s, cell_old, xnew, r.yi);
    uint32_t newloc = r.iloc;
    if (cell_new != cell_old) {
        // the new cell lies in the active disk's row of the scanned footprint,
        // whose empty slots the scan recorded (else they are read here)
        int mc = (int)(cell_new % (uint32_t)s.nc) - o.cx;
        if (mc < 0) mc += s.nc;
        unsigned em;
        if (mc <= o.mlast && (mc + 1) * C <= 64) {
            em = (unsigned)(o.emask >> (mc * C)) & ((1u << C) - 1u);
        } else {
            const uint32_t sid = (lane < C) ? s.cid[cell_new * C + lane] : 0u;
            em = __ballot_sync(FULL, lane < C && sid == EMPTY);
        }
        if (!em) return EMPTY;
        newloc = cell_new * C + (uint32_t)(__ffs(em) - 1);
        if (lane == 0) {
            s.cx[newloc] = xnew;
            s.cy[newloc] = r.yi;
            if (s.cskp) s.cskp[newloc] = (uint8_t)r.skip;
            s.ct[newloc] = tnew;
            s.cown[newloc] = own_new;
            s.cid[newloc] = r.i;
            s.cid[r.iloc] = EMPTY;
        }
    } else if (lane == 0) {
        s.cx[r.iloc] = xnew;
        s.ct[r.iloc] = tnew;
        s.cown[r.iloc] = own_new;
    }
    return newloc;
}

// Executes a step (a lifting, Eq. 1, or a stall at the breakpoint) and returns the
// chain's new status; *newloc receives the moved disk's slot. Writes are done
// by lane 0; all lanes update the registers. In pass 1 the owner word of the
// target is taken with atomicCAS whose result (*cas_old, lane 0) the caller
// checks later; in repair the component owns every cell it touches.
template <int C>
__device__ int commit_step(const Dev &s, int c, ChainReg &r, const StepOut &o, bool pass1,
                           uint32_t seq, int32_t nrec, uint32_t *newloc_out, uint32_t *cas_old) {
    const int lane = threadIdx.x & 31;
    if (nrec >= s.cap) {
        if (lane == 0) atomicAdd(s.lc + LC_ERR_REC, 1ull);
        return ST_BLOCKED;
    }
    if (o.lift) {
        // local times before the position (Remark 11)
        const double tnew = __dadd_rn(r.ti, o.tau);      // new t_j = new t_i
        const double xnew = wrap_add(r.xi, o.tau, s);    // i moves to contact
        if (lane == 0) {
            if (pass1)
                *cas_old = atomicCAS(s.cown + o.jloc, OWN_STATIC, OWN_ACTIVE | (uint32_t)c);
            else
                s.cown[o.jloc] = OWN_ACTIVE | (uint32_t)c;
            s.ct[o.jloc] = tnew;
        }
        const uint32_t newloc = move_active<C>(s, r, o, xnew, tnew, OWN_STATIC);  // i static
        if (newloc == EMPTY) {
            if (lane == 0) atomicAdd(s.lc + LC_ERR_CAP, 1ull);
            return ST_BLOCKED;
        }
        if (lane == 0) {
            Rec q;
            q.i = r.i;
            q.from = r.iloc;
            q.to = newloc;
            q.j = o.j;
            q.jloc = o.jloc;
            q.seq = seq;
            q.flags = 0;
            q.pad = 0;
            q.x_old = r.xi;
            q.ti_old = r.ti;
            q.tj_old = o.tj;
            q.t = tnew;
            q.tau = o.tau;
            q.xi = xnew;
            q.xj = o.xj;
            q.d_after = __dsub_rn(r.D, o.tau);
            *rec_at(s, c, nrec) = q;
            s.nrec[c] = nrec + 1;
            atomicAdd(s.nlift + c, 1);
        }
        *newloc_out = newloc;
        r.D = __dsub_rn(r.D, o.tau);                     // remaining length
        r.i = o.j;                                       // activity passes to j
        r.iloc = o.jloc;
        r.xi = o.xj;
        r.yi = o.yj;
        r.ti = tnew;
        // (pass 1 gathered them with the target's slot)
        r.skip = pass1 ? o.jskp : skip_of(s, o.jloc);
        __syncwarp();
        return ST_RUNNING;
    }
    const double tnew = __dadd_rn(r.ti, r.D);           // t_i reaches the breakpoint
    const double xnew = wrap_add(r.xi, r.D, s);         // i moves by D
    const uint32_t newloc = move_active<C>(s, r, o, xnew, tnew, OWN_STALLED | (uint32_t)c);
    if (newloc == EMPTY) {
        if (lane == 0) atomicAdd(s.lc + LC_ERR_CAP, 1ull);
        return ST_BLOCKED;
    }
    if (lane == 0) {
        Rec q;
        q.i = r.i;
        q.from = r.iloc;
        q.to = newloc;
        q.j = NONE;
        q.jloc = 0;
        q.seq = seq;
        q.flags = 0;
        q.pad = 0;
        q.x_old = r.xi;
        q.ti_old = r.ti;
        q.tj_old = 0.0;
        q.t = tnew;
        q.tau = r.D;
        q.xi = xnew;
        q.xj = 0.0;
        q.d_after = 0.0;
        *rec_at(s, c, nrec) = q;
        s.nrec[c] = nrec + 1;
    }
    *newloc_out = newloc;
    r.iloc = newloc;
    r.xi = xnew;
    r.ti = tnew;
    r.D = 0.0;                                          // stalled
    __syncwarp();
    return ST_STALLED;
}

// A chain blocked by the window's parallel pass (lane 0): counted, listed for
// the union-find, and counted against its partner.
__device__ __forceinline__ void note_blocked(const Dev &s, int c, int32_t partner) {
    atomicAdd(s.lc + LC_BLOCKED, 1ull);
    const unsigned long long ix = atomicAdd(s.lc + LC_WBLOCKED, 1ull);
    if (ix < (unsigned long long)s.k) s.blist[ix] = c;
    if (partner >= 0 && partner < s.k) atomicAdd(s.pcnt + partner, 1);
}

#include "rowpass.cuh"

// ---------------------------------------------------------------- kernels

// Cells from positions, in two passes (slot order is irrelevant to every
// result). k_place puts each disk's id into a free slot of its cell (a
// compare-and-swap per disk, from slot 0; cid must hold EMPTY) and, with
// bad_xy, counts coordinates outside [0, L). k_fill then writes every slot's
// fields row by row -- whole 32-byte sectors, the slots of a cell by
// consecutive threads -- and each disk's slot into loc_of. (Writing a disk's
// fields from its own thread scattered partial-sector writes over the arrays,
// one per field: about four times the time of both passes.)
template <int C>
__global__ void k_place(Dev s, const double *x, const double *y, unsigned long long *bad_xy) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s.n) return;
    const double xq = x[q], yq = y[q];
    if (bad_xy && !(xq >= 0.0 && xq < s.L && yq >= 0.0 && yq < s.L)) atomicAdd(bad_xy, 1ull);
    const uint32_t cell = cell_of(xq, yq, s);
    for (int sl = 0; sl < C; ++sl)
        if (atomicCAS(s.cid + cell * C + sl, EMPTY, (uint32_t)q) == EMPTY) return;
    atomicAdd(s.lc + LC_ERR_CAP, 1ull);
}

// Kernels over the slots of every cell row take a 2D grid (rows_grid): y the
// cell row, x the 256-slot chunk of the row, one thread per slot -- the row
// without a 64-bit division, and every slot's loads in flight at once.
constexpr int ROW_THREADS = 256;
static dim3 rows_grid(int nc, int C) {
    return dim3((unsigned)(((int64_t)nc * C + ROW_THREADS - 1) / ROW_THREADS), (unsigned)nc);
}

// An empty slot's fields are never read; they are written all the same, so
// that every sector is written whole.
template <int C>
__global__ void __launch_bounds__(ROW_THREADS)
k_fill(Dev s, const double *x, const double *y, uint32_t *loc_of) {
    const uint32_t nrow = (uint32_t)s.nc * C;
    const uint32_t o = blockIdx.x * ROW_THREADS + threadIdx.x;
    if (o >= nrow) return;
    const uint32_t q = blockIdx.y * nrow + o;
    const uint32_t id = s.cid[q];
    double xv = 0.0, yv = 0.0;
    if (id != EMPTY) {
        xv = x[id];
        yv = y[id];
        loc_of[id] = q;
    }
    s.cx[q] = xv;
    s.cy[q] = yv;
    s.ct[q] = 0.0;
    s.cown[q] = OWN_STATIC;
}

template <int C>
static void launch_cells(const Dev &s, const double *x, const double *y, uint32_t *loc_of,
                         unsigned long long *bad_xy, cudaStream_t st) {
    k_place<C><<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s, x, y, bad_xy);
    k_fill<C><<<rows_grid(s.nc, C), ROW_THREADS, 0, st>>>(s, x, y, loc_of);
}

// Least and largest y of each cell row, then the rows a disk's scan need not
// read (Dev::cskp). Take a disk in row R with 1 <= R <= nc - 2 and nc >= 5, so
// that rows R - 1 and R + 1 do not wrap and the scan's |dy| is the plain
// difference (its periodic image is farther); the edge rows follow k_skip.
// - It skips row R + 1 when RN(ylo(R + 1) - y) >= d. Every disk j there has
//   y_j >= ylo, so the scan's |RN(y_j - y)| = RN(y_j - y) >= RN(ylo - y) >= d
//   (rounding is monotone), and j lies in no corridor.
// - It skips row R - 1 when RN(y - yhi(R - 1)) >= d, by the same argument.
// An empty row is skipped. Moves along x never change a disk's row, so the
// bits hold until the frame is transposed.
__global__ void k_band_init(Dev s) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s.nc) return;
    s.rband[q] = INF_BITS;
    s.rband[s.nc + q] = 0ull;
}

// Over rows_grid: each block reduces its chunk of one row and its thread 0
// folds that into the row's band (a few atomics per row, after k_band_init).
__global__ void __launch_bounds__(ROW_THREADS) k_bands(Dev s, int C) {
    __shared__ unsigned long long wlo[ROW_THREADS / 32], whi[ROW_THREADS / 32];
    const uint32_t nrow = (uint32_t)s.nc * (uint32_t)C;
    const uint32_t o = blockIdx.x * ROW_THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long lo = INF_BITS, hi = 0ull;
    if (o < nrow) {
        const uint32_t q = blockIdx.y * nrow + o;
        if (s.cid[q] != EMPTY) {
            const unsigned long long y = dbits(s.cy[q]);  // y >= 0: bits order like values
            lo = y;
            hi = y;
        }
    }
#pragma unroll
    for (int k2 = 16; k2 > 0; k2 >>= 1) {
        const unsigned long long l2 = shfl_xor_u64(lo, k2), h2 = shfl_xor_u64(hi, k2);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if (lane == 0) {
        wlo[w] = lo;
        whi[w] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < ROW_THREADS / 32; ++q) {
            lo = wlo[q] < lo ? wlo[q] : lo;
            hi = whi[q] > hi ? whi[q] : hi;
        }
        if (lo != INF_BITS) {
            atomicMin(s.rband + blockIdx.y, lo);
            atomicMax(s.rband + s.nc + blockIdx.y, hi);
        }
    }
}

// In the edge rows (R = 0 below, R = nc - 1 above) the neighbour row lies
// across the box edge, and the scan takes the periodic image: for j in row
// nc - 1 seen from row 0 its |dy| is RN(L - RN(y_j - y)), which only grows as
// y_j falls, so RN(L - RN(yhi(nc - 1) - y)) >= d bounds the whole row; from row
// nc - 1 towards row 0 it is RN(L - RN(y - y_j)), bounded by RN(L - RN(y -
// ylo(0))). (The plain difference there is close to L, far above d.)
// Over rows_grid, one thread per slot. The occupied slots of the block are
// packed first, so that the FP64 tests run on full warps (an FP64 warp
// instruction occupies the unit as long whatever its lane mask, and most
// slots are empty: one disk per cell of four slots on a lattice).
__global__ void __launch_bounds__(ROW_THREADS) k_skip(Dev s, int C) {
    __shared__ uint32_t occ_q[ROW_THREADS];
    __shared__ int n_occ;
    const int nc = s.nc, R = (int)blockIdx.y;
    const uint32_t nrow = (uint32_t)nc * (uint32_t)C;
    const int Rdn = R == 0 ? nc - 1 : R - 1, Rup = R == nc - 1 ? 0 : R + 1;
    const unsigned long long lo_dn = s.rband[Rdn], lo_up = s.rband[Rup];
    const double hi_dn = __longlong_as_double((long long)s.rband[nc + Rdn]);
    const double lo = __longlong_as_double((long long)lo_up);
    const uint32_t o = blockIdx.x * ROW_THREADS + threadIdx.x;
    if (threadIdx.x == 0) n_occ = 0;
    __syncthreads();
    if (o < nrow) {
        const uint32_t q = (uint32_t)R * nrow + o;
        if (s.cid[q] != EMPTY && nc >= 5)
            occ_q[atomicAdd(&n_occ, 1)] = q;
        else
            s.cskp[q] = 0;
    }
    __syncthreads();
    if ((int)threadIdx.x < n_occ) {
        const uint32_t q = occ_q[threadIdx.x];
        uint8_t v = 0;
        {
            const double y = s.cy[q];
            if (lo_dn == INF_BITS) {
                v |= 1;
            } else if (R == 0) {
                if (!(__dsub_rn(s.L, __dsub_rn(hi_dn, y)) < s.d)) v |= 1;
            } else if (!(__dsub_rn(y, hi_dn) < s.d)) {
                v |= 1;
            }
            if (lo_up == INF_BITS) {
                v |= 2;
            } else if (R == nc - 1) {
                if (!(__dsub_rn(s.L, __dsub_rn(y, lo)) < s.d)) v |= 2;
            } else if (!(__dsub_rn(lo, y) < s.d)) {
                v |= 2;
            }
        }
        s.cskp[q] = v;
    }
}

// Skip bits for the current frame (after the cells are built or transposed).
static void launch_skip(const Dev &s, int C, cudaStream_t st) {
    k_band_init<<<(unsigned)((s.nc + 255) / 256), 256, 0, st>>>(s);
    k_bands<<<rows_grid(s.nc, C), ROW_THREADS, 0, st>>>(s, C);
    k_skip<<<rows_grid(s.nc, C), ROW_THREADS, 0, st>>>(s, C);
}

// Coordinates in [0, L) (counted in *bad_xy; not checked with x == null) and
// distinct active ids in [0, n) (*bad_id), checked on the device where the
// inputs already are. seen[] must be zero.
__global__ void k_check_inputs(const double *x, const double *y, const int32_t *active,
                               int64_t n, int k, double L, uint32_t *seen,
                               unsigned long long *bad_xy, unsigned long long *bad_id) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t q = t0; x && q < n; q += stride)
        if (!(x[q] >= 0.0 && x[q] < L && y[q] >= 0.0 && y[q] < L)) atomicAdd(bad_xy, 1ull);
    for (int64_t c = t0; c < k; c += stride) {
        const int32_t a = active[c];
        if (a < 0 || (int64_t)a >= n || atomicExch(seen + a, 1u) != 0u) atomicAdd(bad_id, 1ull);
    }
}

static void launch_check(const double *x, const double *y, const int32_t *active, int64_t n,
                         int k, double L, uint32_t *seen, unsigned long long *bad_xy,
                         unsigned long long *bad_id, cudaStream_t st) {
    const int64_t work = x ? std::max<int64_t>(n, k) : (int64_t)k;
    const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, 4096);
    k_check_inputs<<<blocks, 256, 0, st>>>(x, y, active, n, k, L, seen, bad_xy, bad_id);
}

__global__ void k_init_chains(Dev s, const int32_t *active, const uint32_t *loc_of) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.k || s.lc[LC_BADID] != 0ull) return;  // ids checked before, in stream order
    const uint32_t a = (uint32_t)active[c];
    const uint32_t loc = loc_of[a];
    s.aloc[c] = loc;
    s.ci[c] = a;
    s.cown[loc] = OWN_ACTIVE | (uint32_t)c;
    s.nrec[c] = 0;
    s.status[c] = ST_STALLED;
}

// Leg start: clear local times left by the previous leg (every slot a record
// names), then start every chain on its stalled disk with D = ell (Alg. 2
// input at h).
__device__ void leg_begin_chain(const Dev &s, int c) {
    // (fields held in registers: the global Dev would be re-read after every
    // store)
    const int32_t nr = s.nrec[c];
    double *const ct = s.ct;
    // records read 8 at a time before their stores (a store between two loads
    // could alias the next record and would serialise the round trips)
    for (int32_t e0 = 0; e0 < nr; e0 += 8) {
        uint32_t to[8], jl[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            to[u] = EMPTY;
            jl[u] = EMPTY;
            if (e0 + u < nr) {
                const Rec *q = rec_at(s, c, e0 + u);
                to[u] = q->to;
                if (q->j != NONE) jl[u] = q->jloc;
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (to[u] != EMPTY) ct[to[u]] = 0.0;
            if (jl[u] != EMPTY) ct[jl[u]] = 0.0;
        }
    }
    const uint32_t loc = s.aloc[c];
    uint32_t *const cown = s.cown;
    const uint32_t id = s.cid[loc];
    const double ell = s.ell;
    uint32_t *const ci = s.ci, *const aloc0 = s.aloc0;
    double *const D = s.D, *const tc = s.tc;
    int32_t *const status = s.status, *const partner = s.partner, *const nrec = s.nrec,
                   *const nlift = s.nlift;
    cown[loc] = OWN_ACTIVE | (uint32_t)c;
    ci[c] = id;
    aloc0[c] = loc;
    D[c] = ell;
    tc[c] = 0.0;
    status[c] = ST_RUNNING;
    partner[c] = -1;
    nrec[c] = 0;
    nlift[c] = 0;
}

__global__ void k_leg_begin(Dev s) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < s.k) leg_begin_chain(s, c);
}

// leg_begin_chain by a warp: the lanes clear the local times of the chain's
// records in parallel (one round trip for up to 32 records), lane 0 sets the
// chain table. Returns (on lane 0) whether the table named the disk that its
// active slot holds (the chain-table invariant).
__device__ bool leg_begin_chain_warp(const Dev &s, int c, int lane) {
    const int32_t nr = s.nrec[c];
    double *const ct = s.ct;
    for (int32_t e = lane; e < nr; e += 32) {
        const Rec *q = rec_at(s, c, e);
        const uint32_t to = q->to, j = q->j, jl = q->jloc;
        ct[to] = 0.0;
        if (j != NONE) ct[jl] = 0.0;
    }
    bool ok = true;
    if (lane == 0) {
        const uint32_t loc = s.aloc[c];
        const uint32_t id = s.cid[loc];
        const uint32_t id_was = s.ci[c];
        ok = id == id_was;
        s.cown[loc] = OWN_ACTIVE | (uint32_t)c;
        s.ci[c] = id;
        s.aloc0[c] = loc;
        s.D[c] = s.ell;
        s.tc[c] = 0.0;
        s.status[c] = ST_RUNNING;
        s.partner[c] = -1;
        s.nrec[c] = 0;
        s.nlift[c] = 0;
    }
    __syncwarp();
    return ok;
}

// Pass 1 of a claim window [tw, tend): one warp runs chain c from its current
// state through its events before tend, until it stalls, pauses at tend or
// meets a conflict.
template <int C>
__device__ void pass1_chain(const Dev &s, int c, double tw, double tend) {
    const int lane = threadIdx.x & 31;
    if (s.status[c] != ST_RUNNING) return;
    ChainReg r;
    r.iloc = s.aloc[c];
    r.i = s.ci[c];
    if (lane == 0 && (s.cid[r.iloc] != r.i || s.cown[r.iloc] != (OWN_ACTIVE | (uint32_t)c)))
        diag(s, 6, tw, c, r.i, s.cid[r.iloc], s.cown[r.iloc], s.tc[c]);
    r.xi = s.cx[r.iloc];
    r.yi = s.cy[r.iloc];
    r.ti = s.tc[c];
    r.D = s.D[c];
    r.skip = skip_of(s, r.iloc);
    int st = ST_RUNNING;
    uint32_t seq = (uint32_t)s.nrec[c];
    bool weak = false;  // the claim sets met on a weak claim
    uint32_t cas_old = OWN_STATIC;  // lane 0: owner word seen by the last lift's CAS
    int32_t cas_rec = -1;           // record of that lift, while unchecked
    bool blocked = false;
    uint32_t lifts = 0;
    while (st == ST_RUNNING) {
        const StepOut o = scan_step<C, MODE_PASS1>(s, c, c, r, tw);
        weak |= o.weak != 0;
        if (cas_rec >= 0) {  // the CAS ran while this step's cells were loaded
            const uint32_t old = __shfl_sync(FULL, cas_old, 0);
            if (old != OWN_STATIC) {
                // the owner word was read as static in a cell this chain holds,
                // so no other chain can have taken it: kept as a check that
                // blocks the chain (and names the owner) should it ever fail
                if (lane == 0) {
                    rec_at(s, c, cas_rec)->flags |= REC_NO_OWNER;
                    s.partner[c] = (int32_t)(old & OWN_CHAIN);
                    atomicAdd(s.lc + LC_OWNER_FAIL, 1ull);
                }
                blocked = true;
                break;
            }
            cas_rec = -1;
        }
        if (o.conflict) {
            if (lane == 0) s.partner[c] = (int32_t)o.partner;
            blocked = true;
            break;
        }
        if (o.nonstatic) {
            // Alg. 4 would lift onto another chain's disk (Remark 10): stop
            // here, in one component with that chain (whose claims overlap)
            if (lane == 0) s.partner[c] = o.ns_owner < (uint32_t)s.k ? (int32_t)o.ns_owner : -1;
            blocked = true;
            break;
        }
        if (!(dbits(__dadd_rn(r.ti, o.tau)) < dbits(tend))) break;  // pauses at the window end
        if (dbits(__dadd_rn(r.ti, o.tau)) < dbits(tw) && lane == 0) {
            // a window's events start at its start time (repairs roll back to it)
            atomicAdd(s.lc + LC_ORDER, 1ull);
            diag(s, 9, tw, c, r.i, o.j, r.ti, o.tau);
        }
        uint32_t nl;
        st = commit_step<C>(s, c, r, o, true, seq, (int32_t)seq, &nl, &cas_old);
        if (st == ST_RUNNING) {
            cas_rec = (int32_t)seq;
            ++lifts;
        }
        ++seq;
    }
    if (blocked) st = ST_BLOCKED;
    if (lane == 0) {
        // events before the blocking time, and all before the window, are exact
        s.vt[c] = blocked ? fmax(r.ti, tw) : INFINITY;
        s.status[c] = st;
        s.aloc[c] = r.iloc;
        s.ci[c] = r.i;
        s.tc[c] = r.ti;
        s.D[c] = r.D;
        if (blocked) note_blocked(s, c, s.partner[c]);
        if (weak) {
            atomicAdd(s.lc + LC_WEAK, 1ull);
            atomicAdd(s.lc + LC_WWEAK, 1ull);
        }
        atomicAdd(s.lc + LC_P1LIFTS, (unsigned long long)lifts);
    }
    __syncwarp();
}

template <int C>
__global__ void k_pass1(Dev s) {
    const int warps = blockDim.x >> 5;
    const int c = blockIdx.x * warps + (threadIdx.x >> 5);
    if (c < s.k) pass1_chain<C>(s, c, 0.0, INFINITY);
}

// Exact inverse of commit_step for one record of chain c (one lane).
__device__ void undo_record(const Dev &s, int c, const Rec &u) {
    if (u.to != u.from) {
        s.cx[u.from] = u.x_old;
        s.cy[u.from] = s.cy[u.to];
        if (s.cskp) s.cskp[u.from] = s.cskp[u.to];
        s.cid[u.from] = u.i;
        s.cid[u.to] = EMPTY;
    } else {
        s.cx[u.from] = u.x_old;
    }
    s.ct[u.from] = u.ti_old;
    s.cown[u.from] = OWN_ACTIVE | (uint32_t)c;
    if (u.j != NONE) {
        s.ct[u.jloc] = u.tj_old;
        if (!(u.flags & REC_NO_OWNER)) s.cown[u.jloc] = OWN_STATIC;
        atomicSub(s.nlift + c, 1);
    }
}

__global__ void k_uf(Dev s, int first) {
    __shared__ int warp_tot[32];
    __shared__ int tot[2];
    uf_block(s, first, warp_tot, tot, true);
}

__device__ __forceinline__ bool footprint_has(int fcx, int fcy, int fm, uint32_t cell, int nc) {
    const int r = (int)(cell / (uint32_t)nc), col = (int)(cell % (uint32_t)nc);
    int dr = r - fcy;
    if (dr < 0) dr += nc;
    if (!(dr == 0 || dr == 1 || dr == nc - 1)) return false;
    int dm = col - fcx;
    if (dm < 0) dm += nc;
    return dm <= fm;
}

// Rolls the members of a component back to T* (their events before T* are
// exact): records with event time >= T* are undone, latest first. Records of
// repair rounds (seq >= REPAIR_SEQ0) can share slots across members and are
// undone one at a time in descending seq; beneath them, the records of the
// window's pass 1 lie in cells claimed by their own chain only, so each
// member undoes its own in parallel.
__device__ void rollback_members(const Dev &s, const int32_t *mem, int m, double Ts) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t bseq = 0;
        int bmem = -1;
        for (int e = lane; e < m; e += 32) {
            const int c = mem[e];
            const int32_t nr = s.nrec[c];
            if (nr == 0) continue;
            const Rec &u = *rec_at(s, c, nr - 1);
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
            undo_record(s, c, *rec_at(s, c, nr - 1));
            s.nrec[c] = nr - 1;
        }
        __syncwarp();
    }
    for (int e = lane; e < m; e += 32) {
        const int c = mem[e];
        int32_t nr = s.nrec[c];
        while (nr > 0) {
            const Rec &u = *rec_at(s, c, nr - 1);
            if (!(u.t >= Ts)) break;
            undo_record(s, c, u);
            --nr;
        }
        s.nrec[c] = nr;
    }
    __syncwarp();
}

// State of chain c after its last kept record (or at the leg start).
__device__ void resume_state(const Dev &s, int c, uint32_t &loc, uint32_t &id, double &t,
                             double &D, int &st) {
    const int32_t nr = s.nrec[c];
    if (nr == 0) {
        loc = s.aloc0[c];
        id = s.cid[loc];
        t = 0.0;
        D = s.ell;
        st = ST_RUNNING;
        return;
    }
    const Rec &u = *rec_at(s, c, nr - 1);
    if (u.j == NONE) {
        loc = u.to;
        id = u.i;
        t = u.t;
        D = 0.0;
        st = ST_STALLED;
    } else {
        loc = u.jloc;
        id = u.j;
        t = u.t;
        D = u.d_after;
        st = ST_RUNNING;
    }
}

// After a component's redo: record abort or success for the next round.
// keep_vt (success): the members' vt becomes `now` instead of infinity, so
// that a later merge rolls them back to `now` or earlier (their slot
// operations were not applied in time order, so none may stay on top of an
// undone earlier one).
__device__ void finish_component(const Dev &s, const int32_t *mem, int m, int root, bool abort,
                                 int met, double now, bool keep_vt = false) {
    const int lane = threadIdx.x & 31;
    if (abort) {
        // events before `now` are exact; the chain met joins next round
        for (int e = lane; e < m; e += 32) s.vt[mem[e]] = now;
        if (lane == 0) {
            if (met >= 0) {
                s.abort_to[root] = met;
                atomic_min_time(s.vt + met, now);
            }
            atomicAdd(s.ctl + CTL_NABORT, 1);
        }
    } else {
        for (int e = lane; e < m; e += 32) {
            s.fin[mem[e]] = 2;
            s.vt[mem[e]] = keep_vt ? now : INFINITY;
        }
    }
    __syncwarp();
}

// Redo of a component with at most 32 members: member e's state and pending
// event live in the registers of lane e.
template <int C>
__device__ void repair_small(const Dev &s, const int32_t *mem, int m, int root, double Ts,
                             int round, double tend) {
    const int lane = threadIdx.x & 31;
    const bool has = lane < m;
    const int my_c = has ? mem[lane] : 0x7FFFFFFF;
    uint32_t my_loc = 0, my_id = 0, my_skp = 0;
    double my_x = 0.0, my_y = 0.0, my_t = 0.0, my_D = 0.0;
    int my_st = ST_STALLED;
    int32_t my_nrec = 0;
    if (has) {
        resume_state(s, my_c, my_loc, my_id, my_t, my_D, my_st);
        my_nrec = s.nrec[my_c];
        my_x = s.cx[my_loc];
        my_y = s.cy[my_loc];
        my_skp = skip_of(s, my_loc);
        if (s.cid[my_loc] != my_id) {
            const int32_t nr = s.nrec[my_c];
            diag(s, 1, round, my_c, my_loc, my_id, s.cid[my_loc],
                 nr > 0 ? (double)rec_at(s, my_c, nr - 1)->seq : -1.0);
        }
    }
    // pending event
    unsigned long long ev_T = INF_BITS;
    StepOut ev;
    ev.lift = 0;
    ev.tau = 0.0;
    ev.j = NONE;
    ev.jloc = 0;
    ev.xj = ev.yj = ev.tj = 0.0;
    ev.cx = ev.cy = 0;
    ev.mlast = -1;
    ev.emask = 0ull;
    ev.nonstatic = ev.viol = 0;
    bool abort = false;
    int met = -1;
    // computes member q's next event into lane q's registers
    auto compute = [&](int q) {
        ChainReg r;
        r.i = __shfl_sync(FULL, my_id, q);
        r.iloc = __shfl_sync(FULL, my_loc, q);
        r.xi = __shfl_sync(FULL, my_x, q);
        r.yi = __shfl_sync(FULL, my_y, q);
        r.skip = __shfl_sync(FULL, my_skp, q);
        r.ti = __shfl_sync(FULL, my_t, q);
        r.D = __shfl_sync(FULL, my_D, q);
        const int cq = __shfl_sync(FULL, my_c, q);
        const StepOut o = scan_step<C, MODE_COMP>(s, cq, root, r, 0.0, m, my_c);
        if (o.conflict) {
            abort = true;
            met = (int)o.partner;
        }
        if (lane == q) {
            ev = o;
            ev_T = dbits(__dadd_rn(r.ti, o.tau));
        }
    };
    {
        unsigned b = __ballot_sync(FULL, has && my_st == ST_RUNNING);
        while (b && !abort) {
            const int q = __ffs(b) - 1;
            b &= b - 1;
            compute(q);
        }
    }
    double now = Ts;
    uint32_t cnt = 0;
    while (!abort) {
        unsigned long long bT = (has && my_st == ST_RUNNING) ? ev_T : ~0ull;
        int bc = (has && my_st == ST_RUNNING) ? my_c : 0x7FFFFFFF;
        int bq = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long T2 = shfl_xor_u64(bT, o);
            const int c2 = __shfl_xor_sync(FULL, bc, o);
            const int q2 = __shfl_xor_sync(FULL, bq, o);
            if (T2 < bT || (T2 == bT && c2 < bc)) {
                bT = T2;
                bc = c2;
                bq = q2;
            }
        }
        if (bc == 0x7FFFFFFF) break;
        if (!(bT < dbits(tend))) break;  // the rest lies in a later window
        const double Tn = __longlong_as_double((long long)bT);
        if (dbits(Tn) < dbits(now) && lane == 0) {
            atomicAdd(s.lc + LC_ORDER, 1ull);
            diag(s, 2, round, bc, Tn, now, Ts, m);
        }
        now = Tn;
        ChainReg r;
        r.i = __shfl_sync(FULL, my_id, bq);
        r.iloc = __shfl_sync(FULL, my_loc, bq);
        r.xi = __shfl_sync(FULL, my_x, bq);
        r.yi = __shfl_sync(FULL, my_y, bq);
        r.skip = __shfl_sync(FULL, my_skp, bq);
        r.ti = __shfl_sync(FULL, my_t, bq);
        r.D = __shfl_sync(FULL, my_D, bq);
        StepOut o;
        o.lift = __shfl_sync(FULL, ev.lift, bq);
        o.tau = __shfl_sync(FULL, ev.tau, bq);
        o.j = __shfl_sync(FULL, ev.j, bq);
        o.jloc = __shfl_sync(FULL, ev.jloc, bq);
        o.xj = __shfl_sync(FULL, ev.xj, bq);
        o.yj = __shfl_sync(FULL, ev.yj, bq);
        o.tj = __shfl_sync(FULL, ev.tj, bq);
        o.cx = __shfl_sync(FULL, ev.cx, bq);
        o.mlast = __shfl_sync(FULL, ev.mlast, bq);
        o.emask = shfl_u64(ev.emask, bq);
        const uint32_t cell_a = r.iloc / C;
        const uint32_t cell_j = o.lift ? o.jloc / C : cell_a;
        uint32_t nl = 0, dummy = 0;
        const double y_moved = r.yi;  // the moved disk keeps its y
        const int st = commit_step<C>(s, bc, r, o, false, ((uint32_t)round << 24) | cnt++,
                                      __shfl_sync(FULL, my_nrec, bq), &nl, &dummy);
        if (st == ST_BLOCKED) {  // out of records or slots: reported by the host
            abort = true;
            break;
        }
        const uint32_t cell_b = nl / C;
        if (lane == bq) {
            my_nrec += 1;
            my_st = st;
            my_loc = r.iloc;
            my_id = r.i;
            my_x = r.xi;
            my_y = r.yi;
            my_skp = r.skip;
            my_t = r.ti;
            my_D = r.D;
        }
        // a member's pending event can change only through a disk in its
        // corridor (|dy| < d from its active disk), or through the empty slots
        // of its active disk's row (where it will move)
        auto near = [&](double y) {
            double a = fabs(__dsub_rn(y, my_y));
            if (dbits(__dsub_rn(s.L, a)) < dbits(a)) a = __dsub_rn(s.L, a);
            return dbits(a) < dbits(s.d);
        };
        auto in_row = [&](uint32_t cell) {
            return (int)(cell / (uint32_t)s.nc) == ev.cy &&
                   footprint_has(ev.cx, ev.cy, ev.mlast, cell, s.nc);
        };
        bool redo = false;
        if (has && my_st == ST_RUNNING) {
            if (lane == bq) {
                redo = true;
            } else {
                const bool nm = near(y_moved);
                redo = (footprint_has(ev.cx, ev.cy, ev.mlast, cell_a, s.nc) &&
                        (nm || in_row(cell_a))) ||
                       (footprint_has(ev.cx, ev.cy, ev.mlast, cell_b, s.nc) &&
                        (nm || in_row(cell_b))) ||
                       (o.lift && footprint_has(ev.cx, ev.cy, ev.mlast, cell_j, s.nc) &&
                        near(o.yj));
            }
        }
        unsigned b = __ballot_sync(FULL, redo);
        while (b && !abort) {
            const int q = __ffs(b) - 1;
            b &= b - 1;
            compute(q);
        }
    }
    if (has) {
        s.status[my_c] = my_st;
        s.aloc[my_c] = my_loc;
        s.ci[my_c] = my_id;
        s.tc[my_c] = my_t;
        s.D[my_c] = my_D;
    }
    __syncwarp();
    finish_component(s, mem, m, root, abort, met, now);
}

template <int C>
__device__ StepOut compute_event_global(const Dev &s, int c, int root) {
    const int lane = threadIdx.x & 31;
    ChainReg r;
    r.iloc = s.aloc[c];
    r.i = s.ci[c];
    r.xi = s.cx[r.iloc];
    r.yi = s.cy[r.iloc];
    r.skip = skip_of(s, r.iloc);
    r.ti = s.tc[c];
    r.D = s.D[c];
    const StepOut o = scan_step<C, MODE_COMP>(s, c, root, r, 0.0);
    if (lane == 0) {
        s.ev_T[c] = __dadd_rn(r.ti, o.tau);
        s.ev_tau[c] = o.tau;
        s.ev_j[c] = o.j;
        s.ev_jloc[c] = o.jloc;
        s.ev_xj[c] = o.xj;
        s.ev_yj[c] = o.yj;
        s.ev_tj[c] = o.tj;
        s.ev_lift[c] = o.lift;
        s.ev_cx[c] = o.cx;
        s.ev_cy[c] = o.cy;
        s.ev_mlast[c] = o.mlast;
    }
    __syncwarp();
    return o;
}

// Redo of a component with more than 32 members: state in global memory.
template <int C>
__device__ void repair_large(const Dev &s, const int32_t *mem, int m, int root, double Ts,
                             int round, double tend) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < m; e += 32) {
        const int c = mem[e];
        uint32_t loc, id;
        double t, D;
        int st;
        resume_state(s, c, loc, id, t, D, st);
        if (s.cid[loc] != id) {
            const int32_t nr = s.nrec[c];
            diag(s, 11, round, c, loc, id, s.cid[loc],
                 nr > 0 ? (double)rec_at(s, c, nr - 1)->seq : -1.0);
        }
        s.aloc[c] = loc;
        s.ci[c] = id;
        s.tc[c] = t;
        s.D[c] = D;
        s.status[c] = st;
    }
    __syncwarp();
    bool abort = false;
    int met = -1;
    for (int e = 0; e < m && !abort; ++e) {
        const int c = mem[e];
        if (s.status[c] != ST_RUNNING) continue;
        const StepOut o = compute_event_global<C>(s, c, root);
        if (o.conflict) {
            abort = true;
            met = (int)o.partner;
        }
    }
    double now = Ts;
    uint32_t cnt = 0;
    while (!abort) {
        double bT = INFINITY;
        int bc = 0x7FFFFFFF;
        for (int e = lane; e < m; e += 32) {
            const int c = mem[e];
            if (s.status[c] != ST_RUNNING) continue;
            const double T = s.ev_T[c];
            if (T < bT || (T == bT && c < bc)) {
                bT = T;
                bc = c;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double T2 = __shfl_xor_sync(FULL, bT, o);
            const int c2 = __shfl_xor_sync(FULL, bc, o);
            if (T2 < bT || (T2 == bT && c2 < bc)) {
                bT = T2;
                bc = c2;
            }
        }
        if (bc == 0x7FFFFFFF) break;
        if (!(bT < tend)) break;  // the rest lies in a later window
        if (bT < now && lane == 0) atomicAdd(s.lc + LC_ORDER, 1ull);
        now = bT;
        ChainReg r;
        r.iloc = s.aloc[bc];
        r.i = s.ci[bc];
        r.xi = s.cx[r.iloc];
        r.yi = s.cy[r.iloc];
        r.skip = skip_of(s, r.iloc);
        r.ti = s.tc[bc];
        r.D = s.D[bc];
        StepOut o;
        o.lift = s.ev_lift[bc];
        o.tau = s.ev_tau[bc];
        o.j = s.ev_j[bc];
        o.jloc = s.ev_jloc[bc];
        o.xj = s.ev_xj[bc];
        o.yj = s.ev_yj[bc];
        o.tj = s.ev_tj[bc];
        o.cx = 0;
        o.mlast = -1;  // no recorded empty slots: move_active reads the new cell
        o.emask = 0ull;
        o.nonstatic = o.viol = 0;
        const uint32_t cell_a = r.iloc / C;
        const uint32_t cell_j = o.lift ? o.jloc / C : cell_a;
        uint32_t nl = 0, dummy = 0;
        const int st = commit_step<C>(s, bc, r, o, false, ((uint32_t)round << 24) | cnt++,
                                      s.nrec[bc], &nl, &dummy);
        if (st == ST_BLOCKED) {
            abort = true;
            break;
        }
        const uint32_t cell_b = nl / C;
        if (lane == 0) {
            s.status[bc] = st;
            s.aloc[bc] = r.iloc;
            s.ci[bc] = r.i;
            s.tc[bc] = r.ti;
            s.D[bc] = r.D;
        }
        __syncwarp();
        for (int base = 0; base < m && !abort; base += 32) {
            const int e = base + lane;
            bool redo = false;
            if (e < m) {
                const int c = mem[e];
                if (s.status[c] == ST_RUNNING)
                    redo = c == bc ||
                           footprint_has(s.ev_cx[c], s.ev_cy[c], s.ev_mlast[c], cell_a, s.nc) ||
                           footprint_has(s.ev_cx[c], s.ev_cy[c], s.ev_mlast[c], cell_b, s.nc) ||
                           footprint_has(s.ev_cx[c], s.ev_cy[c], s.ev_mlast[c], cell_j, s.nc);
            }
            unsigned b = __ballot_sync(FULL, redo);
            while (b && !abort) {
                const int q = __ffs(b) - 1;
                b &= b - 1;
                const StepOut o2 = compute_event_global<C>(s, mem[base + q], root);
                if (o2.conflict) {
                    abort = true;
                    met = (int)o2.partner;
                }
            }
        }
    }
    finish_component(s, mem, m, root, abort, met, now);
}

// Component q of the current round: roll its members back to T*, then redo
// them in global event-time order (Alg. 2) while claiming cells for the
// component (one warp).
// First repair round of a claim window: the blocked members continue from
// where they stopped, one after another, over the state the other members
// left. Pass 1 was a run of Alg. 4 (chains advanced one at a time: each
// chain's cells were its own; a chain stopped where Alg. 4 would lift onto
// another chain's disk) in which every step satisfied the horizon condition.
// If every continued step satisfies the horizon condition (Eq. 2) for every
// scanned corridor disk, the whole run is one of Alg. 4 without a horizon
// violation, which by Lemma 2 ends where Alg. 2 ends: nothing has to be
// redone. A member that would lift onto the active disk of another member
// still blocked waits for it (Remark 10): that member continues first.
// Otherwise the caller rolls the component back to T* and replays it in
// global order.
enum { CONT_DONE = 0, CONT_FAIL = 1, CONT_FOREIGN = 2 };

template <int C>
__device__ int continue_component(const Dev &s, const int32_t *mem, int m, int root, int round,
                                  double tw, double tend, int *met) {
    const int lane = threadIdx.x & 31;
    // up to 32 members: members by the lanes' registers, and the component may
    // take over chains that are in no component (the replay that a failure
    // falls back to tests membership against its own member list, so it
    // leaves them alone); more members: by comp_of, no takeover. A failure
    // rolls back to T*: the continued events lie after it, and undoing them
    // all first keeps the slot operations in last-in first-out order.
    const int nm = m <= 32 ? -m : 0;
    const int my_member = lane < m ? mem[lane] : -1;
    // up to 32 members: their status and chain state in one round of loads,
    // one member per lane; the first member continued starts from them (its
    // state is read once instead of after its status)
    int my_st = ST_RUNNING;
    uint32_t my_aloc = 0u, my_ci = 0u;
    double my_tc = 0.0, my_D = 0.0;
    int32_t my_nrec = 0;
    if (nm != 0 && my_member >= 0) {
        my_st = s.status[my_member];
        my_aloc = s.aloc[my_member];
        my_ci = s.ci[my_member];
        my_tc = s.tc[my_member];
        my_D = s.D[my_member];
        my_nrec = s.nrec[my_member];
    }
    bool first = nm != 0;
    uint32_t cnt = 0;
    int e = 0, cur = -1, switches = 0;
    for (;;) {
        if (cur < 0) {  // the next member still blocked
            if (first) {
                const unsigned bm = __ballot_sync(FULL, my_member >= 0 && my_st == ST_BLOCKED);
                if (!bm) break;
                e = __ffs(bm) - 1;
                cur = __shfl_sync(FULL, my_member, e);
            } else {
                while (e < m && s.status[mem[e]] != ST_BLOCKED) ++e;
                if (e >= m) break;
                cur = mem[e];
            }
        }
        const int c = cur;
        int next = -1;
        ChainReg r;
        int32_t nrec;
        if (first) {  // c is the member of lane e
            r.iloc = __shfl_sync(FULL, my_aloc, e);
            r.i = __shfl_sync(FULL, my_ci, e);
            r.ti = __shfl_sync(FULL, my_tc, e);
            r.D = __shfl_sync(FULL, my_D, e);
            nrec = __shfl_sync(FULL, my_nrec, e);
        } else {
            r.iloc = s.aloc[c];
            r.i = s.ci[c];
            r.ti = s.tc[c];
            r.D = s.D[c];
            nrec = s.nrec[c];
        }
        first = false;
        r.xi = s.cx[r.iloc];
        r.yi = s.cy[r.iloc];
        r.skip = skip_of(s, r.iloc);
        int st = ST_RUNNING;
        // members along rows out of reach of their neighbours: the row
        // window while it applies (rowpass.cuh), the general step after
        bool row = s.rp_ok && nm != 0;
        while (st == ST_RUNNING) {
            if (row && r.skip == RP_SKIP_ALL) {
                uint32_t ns_own = NONE;
                const int how = row_cont_member<C>(s, c, round, r, nrec, cnt, tw, tend,
                                                   nm < 0 ? -nm : nm, my_member, st, &ns_own);
                if (how == RC_FAIL) return CONT_FAIL;
                if (how == RC_DONE) break;
                if (how == RC_NONSTATIC) {
                    const int h = (int)ns_own;
                    const bool member = __any_sync(FULL, my_member == h && h >= 0);
                    if (h != c && member && s.status[h] == ST_BLOCKED && switches < 4 * m + 4) {
                        next = h;  // wait for that member
                        st = ST_BLOCKED;
                        ++switches;
                        break;
                    }
                    return CONT_FAIL;
                }
                row = false;  // the general step from here on
            }
            const StepOut o = scan_step<C, MODE_CONT>(s, c, root, r, tw, nm, my_member);
            if (o.conflict) {
                *met = (int)o.partner;
                return CONT_FOREIGN;
            }
            if (o.viol) return CONT_FAIL;
            if (o.nonstatic) {
                const int h = (int)o.ns_owner;
                bool member;
                if (nm != 0)
                    member = __any_sync(FULL, my_member == h && h >= 0);
                else
                    member = h >= 0 && h < s.k && __ldcg(s.comp_of + h) == root;
                if (h != c && member && s.status[h] == ST_BLOCKED && switches < 4 * m + 4) {
                    next = h;  // wait for that member
                    st = ST_BLOCKED;
                    ++switches;
                    break;
                }
                return CONT_FAIL;
            }
            const unsigned long long T = dbits(__dadd_rn(r.ti, o.tau));
            if (!(T < dbits(tend))) break;  // pauses at the window end
            if (T < dbits(tw)) return CONT_FAIL;
            uint32_t nl = 0, unused = 0;
            st = commit_step<C>(s, c, r, o, false, ((uint32_t)round << 24) | cnt++, nrec, &nl,
                                &unused);
            if (st == ST_BLOCKED) return CONT_FAIL;  // out of records or slots
            ++nrec;
        }
        if (lane == 0) {
            s.status[c] = st;
            s.aloc[c] = r.iloc;
            s.ci[c] = r.i;
            s.tc[c] = r.ti;
            s.D[c] = r.D;
        }
        __syncwarp();
        cur = next;
    }
    return CONT_DONE;
}

template <int C>
__device__ void repair_component(const Dev &s, int q, int round, double tw, double tend) {
    const int lane = threadIdx.x & 31;
    const int root = s.comp_root[q];
    const int off = s.comp_off[q], m = s.comp_off[q + 1] - off;
    const int32_t *mem = s.comp_mem + off;
    // T*, the members' earliest time: loaded now, before any member moves, and
    // reduced where it is needed (after the continuation in the first round),
    // so that its loads overlap the continuation's own
    double Ts = INFINITY;
    if (lane < m) Ts = s.vt[mem[lane]];  // (nothing waits on this load yet)
    for (int e = lane + 32; e < m; e += 32) Ts = fmin(Ts, s.vt[mem[e]]);
    auto t_star = [&]() {
        double T = Ts;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) T = fmin(T, __shfl_xor_sync(FULL, T, o));
        return fmax(T, tw);  // earlier windows are final
    };
    if (lane == 0) atomicAdd(s.lc + LC_REPAIRED, (unsigned long long)m);
    if (round == 1) {
        int met = -1;
        const int how = continue_component<C>(s, mem, m, root, round, tw, tend, &met);
        Ts = t_star();
        if (how == CONT_DONE) {
            if (lane == 0) atomicAdd(s.lc + LC_CONTINUED, (unsigned long long)m);
            // a later merge must undo all continued events (they were applied
            // chain by chain, not in time order): it rolls back to T* or earlier
            finish_component(s, mem, m, root, false, -1, Ts, true);
            return;
        }
        if (how == CONT_FOREIGN) {
            // the replay of the merged component rolls back to T* (all of
            // this round's events lie after it)
            finish_component(s, mem, m, root, true, met, Ts);
            return;
        }
    } else {
        Ts = t_star();
    }
    rollback_members(s, mem, m, Ts);
    if (m <= 32)
        repair_small<C>(s, mem, m, root, Ts, round, tend);
    else
        repair_large<C>(s, mem, m, root, Ts, round, tend);
}

template <int C>
__global__ void k_repair(Dev s, int round) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(s.ctl + CTL_WORK, 1);
        q = __shfl_sync(FULL, q, 0);
        if (q >= s.ctl[CTL_NCOMP]) return;
        repair_component<C>(s, q, round, 0.0, INFINITY);
    }
}

// Leg end: totals, and the lifting log (chain by chain).
// Returns the chain's liftings of the leg; count: add them to the leg total
// here (else the caller adds a warp's sum at once).
__device__ int32_t leg_end_chain(const Dev &s, int c, int32_t leg, bool count = true) {
    const int32_t nl = s.nlift[c];
    if (count) atomicAdd(s.lc + LC_LIFTS, (unsigned long long)nl);
    if (s.log_on && nl > 0) {
        const unsigned long long base = atomicAdd(s.tc_cnt + TC_LOG_N, (unsigned long long)nl);
        unsigned long long w = base;
        for (int32_t e = 0; e < s.nrec[c]; ++e) {
            const Rec *q = rec_at(s, c, e);
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
    return nl;
}

__global__ void k_leg_end(Dev s, int32_t leg) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < s.k) leg_end_chain(s, c, leg);
}

template <int C>
__global__ void k_export(Dev s, double *x, double *y, double *t) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)s.nc * s.nc * C) return;
    const uint32_t id = s.cid[q];
    if (id == EMPTY) return;
    if (x) x[id] = s.cx[q];
    if (y) y[id] = s.cy[q];
    if (t) t[id] = s.ct[q];
}

// Direction change at a breakpoint (Sec. 1: in the periodic box the direction
// must change now and then for the algorithm to be irreducible). Motion stays
// +x in the context's frame; moving along +y of the caller's frame is moving
// along +x of the transposed frame, so the context is transposed in place:
// cell (r, c) <-> (c, r), slot for slot, with x and y swapped. Local times are
// cleared (the next leg starts at 0, and the event records that named the
// slots to clear are dropped).
template <int C>
__global__ void k_transpose(Dev s) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)s.nc * s.nc) return;
    const int r = (int)(q / s.nc), c = (int)(q % s.nc);
    if (r > c) return;
    const uint32_t a = (uint32_t)q, b = (uint32_t)c * (uint32_t)s.nc + (uint32_t)r;
    for (int sl = 0; sl < C; ++sl) {
        const uint32_t la = a * C + sl, lb = b * C + sl;
        const double xa = s.cx[la], ya = s.cy[la], xb = s.cx[lb], yb = s.cy[lb];
        const uint32_t ia = s.cid[la], ib = s.cid[lb], oa = s.cown[la], ob = s.cown[lb];
        s.cx[la] = yb;
        s.cy[la] = xb;
        s.cid[la] = ib;
        s.cown[la] = ob;
        s.ct[la] = 0.0;
        s.cx[lb] = ya;
        s.cy[lb] = xa;
        s.cid[lb] = ia;
        s.cown[lb] = oa;
        s.ct[lb] = 0.0;
    }
}

template <int C>
__global__ void k_transpose_chains(Dev s) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.k) return;
    auto tr = [&](uint32_t loc) {
        const uint32_t cell = loc / C, rr = cell / (uint32_t)s.nc, cc = cell % (uint32_t)s.nc;
        return (cc * (uint32_t)s.nc + rr) * C + loc % C;
    };
    s.aloc[c] = tr(s.aloc[c]);
    s.aloc0[c] = tr(s.aloc0[c]);
    s.nrec[c] = 0;
}

__global__ void k_export_active(Dev s, int32_t *active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.k) return;
    active[c] = (int32_t)s.cid[s.aloc[c]];
}

// ------------------------------------------- persistent multi-leg kernel
//
// One cooperative launch runs up to max_legs legs of every live replica
// (independent systems, each with its own Dev). The phases of a leg are
// separated by grid barriers; a replica leaves once it has made its budget of
// liftings. Every barrier wait is bounded by the device clock: past the limit
// the kernel records ECMC_ETIMEOUT and returns instead of waiting on.

struct RepCtl {
    int64_t budget;         // liftings for this run (0: none)
    int64_t lifts;          // liftings made in this run
    int64_t legs;           // legs completed in this run
    int64_t conflict_legs;
    int64_t repaired;
    int64_t continued;
    int64_t horizon;
    int64_t order_err;
    int64_t leg_index0;     // leg index of this run's first leg (lifting log)
    int64_t p1_lifts;       // liftings made by the parallel pass (redone ones included)
    int64_t row_windows;    // claim windows run by the row pass
    int64_t repair_lifts;   // liftings of legs that needed a repair
    int64_t blocked;        // chains whose strong claim was blocked (all windows)
    int64_t cwindows;       // claim windows that needed a repair
    uint8_t *flags;         // per-leg conflict flags (device) or null
    int32_t flags_cap;
    int32_t live;           // takes part in this run
    int32_t done;           // budget reached or error
    int32_t err;            // LC_ERR_* seen
    int32_t incons;         // chain-table checks that failed (must stay 0)
    int32_t bad_where;      // first failure: leg * 65536 + window * 16 + phase
    int32_t bad_chain;
    int32_t dbg;            // an internal check recorded in Dev::dbg (set at the end)
};

enum { G_WORK = 0, G_ANY, G_ERR, G_REMAIN0, G_REMAIN1, G_UFDONE, G_N };
enum { PH_BEGIN = 0, PH_PASS1, PH_REPAIR, PH_END, PH_N };

struct Batch {
    Dev *reps;                    // [R]
    RepCtl *ctl;                  // [R]
    int32_t *chain_base;          // [R+1] prefix of k over replicas
    int32_t *comp_base;           // [R+1] prefix of this round's component counts
    unsigned int *bar;            // [2] grid barrier: arrivals, generation
    int32_t *g;                   // [G_N]
    unsigned long long *phase_ns; // [PH_N] device time per phase (block 0 clock)
    int32_t R;
    int32_t max_legs;
    int32_t windows;  // claim windows per leg (all replicas of a launch)
    int32_t pad;
    unsigned long long wait_ns;  // bound on every grid-barrier wait
};

__device__ __forceinline__ double window_start(const Dev &s, int w) {
    return w == 0 ? 0.0 : __ddiv_rn(__dmul_rn((double)w, s.ell), (double)s.windows);
}

__device__ __forceinline__ double window_end(const Dev &s, int w) {
    return w + 1 >= s.windows ? INFINITY
                              : __ddiv_rn(__dmul_rn((double)(w + 1), s.ell), (double)s.windows);
}

__device__ bool grid_barrier(const Batch &b, int *sflag) {
    return grid_sync(b.bar, b.g + G_ERR, sflag, b.wait_ns);
}

// replica of flattened item w, with base[r] <= w < base[r+1]
__device__ __forceinline__ int find_rep(const int32_t *base, int R, int w) {
    int lo = 0, hi = R;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= w)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool rep_on(const Batch &b, int r) {
    return b.ctl[r].live && !b.ctl[r].done;
}

// A replica with no liftings budget runs every leg of the launch: its next
// leg is begun by its chains at this leg's end (one grid barrier and one pass
// over the chains fewer). With a budget, the leg's totals decide first.
__device__ __forceinline__ bool next_leg_at_end(const Batch &b, int r, int leg) {
    return b.ctl[r].budget == 0 && leg + 1 < b.max_legs;
}

// A thread's index for per-chain loops that spreads consecutive chains over
// the blocks (and so over the SMs): with chains on consecutive threads a few
// blocks would carry all the memory operations of a phase.
__device__ __forceinline__ int spread_index() {
    return (int)(threadIdx.x * gridDim.x + blockIdx.x);
}

// Claim words cleared by the whole grid for the next window (pointers held
// in registers: a field of the global Dev would be re-read after every store).
__device__ __forceinline__ void clear_claims(const Dev &s, int gt, int nthreads) {
    const int64_t ncell = (int64_t)s.nc * s.nc;
    uint32_t *const cl = s.claim;
    for (int64_t q = gt; q < ncell; q += nthreads) cl[q] = 0u;
}

// The row pass's claim arrays, all cells (after a cancelled row pass).
__device__ __forceinline__ void clear_row_claims(const Dev &s, int gt, int nthreads) {
    const int64_t ncell = (int64_t)s.nc * s.nc;
    unsigned long long *const ck = s.ckey;
    uint32_t *const mn = s.camin, *const mx = s.camax;
    for (int64_t q = gt; q < ncell; q += nthreads) {
        ck[q] = ~0ull;
        mn[q] = ~0u;
        mx[q] = 0u;
    }
}

// The system description of the chain (or component) a warp works on, in the
// warp's slot of shared memory: Dev stays constant during a launch, and a
// field read from shared memory costs a few tens of cycles where a read of
// the global copy, which the compiler repeats after every global store, goes
// to L2. rep holds the system whose copy the slot has (-1: none).
__device__ __forceinline__ const Dev &warp_dev(Dev *slot, int *rep, const Dev *reps, int r) {
    if (*(volatile int *)rep != r) {
        constexpr int WORDS = (int)(sizeof(Dev) / sizeof(uint32_t));
        const uint32_t *src = reinterpret_cast<const uint32_t *>(reps + r);
        uint32_t *dst = reinterpret_cast<uint32_t *>(slot);
        for (int q = threadIdx.x & 31; q < WORDS; q += 32) dst[q] = src[q];
        __syncwarp();
        if ((threadIdx.x & 31) == 0) *(volatile int *)rep = r;
        __syncwarp();
    }
    return *slot;
}


// Block shape of the persistent kernel: 8 warps per block, 2 blocks per SM
// (16 warps per SM, 128 registers). Fewer, larger register files (3 blocks of
// 4 warps, no spills) measured slower: the passes want warps more than
// registers.
constexpr int RUN_THREADS = 256;
constexpr int RUN_MIN_BLOCKS = 2;

template <int C>
__global__ void __launch_bounds__(RUN_THREADS, RUN_MIN_BLOCKS) k_run(Batch b) {
    extern __shared__ int32_t uf_sm[];  // UF_SMEM_BYTES: the union-find working set
    __shared__ int warp_tot[32];
    __shared__ int tot[2];
    __shared__ int sflag;
    __shared__ unsigned long long blk_lifts;
    __shared__ Dev wdev[RUN_THREADS / 32];  // per warp: its system's description
    __shared__ int wrep[RUN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wrep[threadIdx.x >> 5] = -1;
    __syncthreads();
    Dev *const my_dev = wdev + (threadIdx.x >> 5);
    int *const my_rep = wrep + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int nwarps = nthreads >> 5;
    const int R = b.R;
    const int total_chains = b.chain_base[R];
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_prev = timer ? gtimer() : 0ull;
    auto mark = [&](int ph) {
        if (timer) {
            const unsigned long long t = gtimer();
            b.phase_ns[ph] += t - t_prev;
            t_prev = t;
        }
    };
    // true in the last block to get here, of all blocks (each block comes
    // once per use): that block finishes a phase's serial tail without a grid
    // barrier before it; it sees every other block's writes of the phase
    auto last_block = [&]() -> bool {
        // (as in the grid barrier: the block barrier, then the master
        // thread's fences, release before the count and acquire after it)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int old = atomicAdd(b.g + G_UFDONE, 1);
            sflag = (old + 1) % (int)gridDim.x == 0;
            if (sflag) __threadfence();
        }
        __syncthreads();
        const bool last = sflag != 0;
        __syncthreads();
        return last;
    };
    // conflict components of replica r (one block): round 1 from the
    // parallel pass's blocked chains, later rounds from the aborts
    auto uf_replica = [&](int r, int round) {
        // the block's copy of the system: warp 0's slot
        if (threadIdx.x < 32) (void)warp_dev(wdev, wrep, b.reps, r);
        __syncthreads();
        const Dev &s = wdev[0];
        bool need = false;
        unsigned long long wbl = 0ull;
        if (rep_on(b, r)) {
            wbl = s.lc[LC_WBLOCKED];
            need = round == 1 ? wbl != 0ull : s.ctl[CTL_NABORT] != 0;
            // the window's flag: the claim sets of two chains met
            if (round == 1 && threadIdx.x == 0 && (wbl != 0ull || s.lc[LC_WWEAK] != 0ull))
                atomicAdd(s.lc + LC_CWINDOWS, 1ull);
        }
        if (need && round <= 255) {
            uf_block(s, round == 1, warp_tot, tot, false, uf_sm, s.blist, s.pcnt,
                     round == 1 ? (int)min(wbl, (unsigned long long)s.k) : -1);
        } else if (threadIdx.x == 0) {
            s.ctl[CTL_NCOMP] = 0;
            if (need) b.ctl[r].err = 1;  // too many rounds
        }
        __syncthreads();
    };
    // prefix of component counts over replicas (one block)
    auto comp_prefix = [&]() {
        const int chunk = (R + blockDim.x - 1) / blockDim.x;
        const int lo = min(R, (int)threadIdx.x * chunk), hi = min(R, lo + chunk);
        int sum = 0;
        for (int r = lo; r < hi; ++r) sum += b.reps[r].ctl[CTL_NCOMP];
        int off = block_exscan(sum, warp_tot, tot);
        for (int r = lo; r < hi; ++r) {
            b.comp_base[r] = off;
            off += b.reps[r].ctl[CTL_NCOMP];
            // every block read the abort counts (the last round's check, this
            // round's need) before it counted itself
            b.reps[r].ctl[CTL_NABORT] = 0;
        }
        if (threadIdx.x == 0) {
            b.comp_base[R] = tot[0];
            b.g[G_WORK] = 0;
            b.g[G_ANY] = tot[0];
        }
    };
    for (int leg = 0; leg < b.max_legs; ++leg) {
        // parity of the row-pass counters of the leg's window w: that of the
        // window's index counted over the launch's legs
        const int p0 = (leg * b.windows) & 1;
        // leg start: chain table, local times, claims, per-leg counters; the
        // chains whose rows are in reach (they rule out the row pass). The
        // replicas whose last leg began this one skip it.
        bool begin_here = false;
        for (int r = 0; r < R; ++r)
            if (rep_on(b, r) && !(leg > 0 && next_leg_at_end(b, r, leg - 1))) begin_here = true;
        if (begin_here) {
            for (int w2 = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; w2 < total_chains;
                 w2 += nwarps) {
                const int r = find_rep(b.chain_base, R, w2);
                if (rep_on(b, r) && !(leg > 0 && next_leg_at_end(b, r, leg - 1))) {
                    const Dev &s = warp_dev(my_dev, my_rep, b.reps, r);
                    const int c = w2 - b.chain_base[r];
                    (void)leg_begin_chain_warp(s, c, lane);
                    if (lane == 0 && s.rp_ok && skip_of(s, s.aloc[c]) != RP_SKIP_ALL)
                        atomicAdd(s.rp + RP_BAD + p0, 1);
                }
            }
            // (claim words were cleared at the end of the last leg, the
            // row-pass counters by its totals)
            for (int r = 0; r < R; ++r)
                if (rep_on(b, r) && !(leg > 0 && next_leg_at_end(b, r, leg - 1)) && gt < LC_N)
                    b.reps[r].lc[gt] = 0ull;
            if (!grid_barrier(b, &sflag)) return;
        }
        mark(PH_BEGIN);
        for (int w = 0; w < b.windows; ++w) {
            const int par = (p0 + w) & 1;
            if (w > 0) {
                // new claim window: claims, the window's blocked count, the
                // chains whose rows are in reach; the other parity's row-pass
                // counters (read in the last window) are cleared
                for (int r = 0; r < R; ++r) {
                    if (!rep_on(b, r)) continue;
                    const Dev &s = b.reps[r];
                    clear_claims(s, gt, nthreads);
                    if (gt == 0) {
                        s.lc[LC_WBLOCKED] = 0ull;
                        s.lc[LC_WWEAK] = 0ull;
                        s.rp[RP_BAD + (par ^ 1)] = 0;
                        s.rp[RP_ABORT + (par ^ 1)] = 0;
                    }
                }
                for (int w2 = spread_index(); w2 < total_chains; w2 += nthreads) {
                    const int r = find_rep(b.chain_base, R, w2);
                    if (!rep_on(b, r)) continue;
                    const Dev &s = b.reps[r];
                    const int c = w2 - b.chain_base[r];
                    if (s.rp_ok && s.status[c] == ST_RUNNING &&
                        skip_of(s, s.aloc[c]) != RP_SKIP_ALL)
                        atomicAdd(s.rp + RP_BAD + par, 1);
                }
                if (!grid_barrier(b, &sflag)) return;
            }
            // parallel pass: one warp per chain, chains spread over the
            // blocks; the row pass where every running chain of the system
            // moves along a row out of reach of its neighbours
            const int lw = threadIdx.x >> 5;
            for (int w2 = lw * gridDim.x + blockIdx.x; w2 < total_chains; w2 += nwarps) {
                const int r = find_rep(b.chain_base, R, w2);
                if (!rep_on(b, r)) continue;
                const Dev &s = warp_dev(my_dev, my_rep, b.reps, r);
                const double tw = window_start(s, w), te = window_end(s, w);
                const int c = w2 - b.chain_base[r];
                if (s.rp_ok && s.rp[RP_BAD + par] == 0) {
                    if (!row_pass_chain<C>(s, c, tw, te) && lane == 0)
                        atomicExch(s.rp + RP_ABORT + par, 1);
                } else {
                    pass1_chain<C>(s, c, tw, te);
                }
            }
            if (!grid_barrier(b, &sflag)) return;
            // the next leg's count of replicas to go (every block has read the
            // last leg's count, the same word, before this barrier)
            if (w == 0 && gt == 0) b.g[G_REMAIN0 + ((leg + 1) & 1)] = 0;
            // row pass: the cells another chain holds, publication, claim
            // words; a cancelled one runs pass1_chain now
            int row_here = 0;
            bool uf_early = false;
            for (int r = threadIdx.x; r < R; r += blockDim.x)
                if (rep_on(b, r) && b.reps[r].rp_ok && b.reps[r].rp[RP_BAD + par] == 0)
                    row_here = 1;
            if (__syncthreads_or(row_here)) {
                for (int w2 = lw * gridDim.x + blockIdx.x; w2 < total_chains; w2 += nwarps) {
                    const int r = find_rep(b.chain_base, R, w2);
                    if (!rep_on(b, r)) continue;
                    const Dev &s = warp_dev(my_dev, my_rep, b.reps, r);
                    if (!(s.rp_ok && s.rp[RP_BAD + par] == 0)) continue;
                    const double tw = window_start(s, w), te = window_end(s, w);
                    const int c = w2 - b.chain_base[r];
                    if (__ldcg(s.rp + RP_ABORT + par) != 0)
                        pass1_chain<C>(s, c, tw, te);
                    else
                        row_resolve_chain<C>(s, c, tw);
                }
                if (R == 1) {
                    // one system: the last block to finish resolving takes
                    // the first round's union-find and prefix (one grid
                    // barrier for both)
                    if (last_block()) {
                        uf_replica(0, 1);
                        comp_prefix();
                    }
                    uf_early = true;
                }
                if (!grid_barrier(b, &sflag)) return;
            }
            mark(PH_PASS1);
            // the row pass's claim arrays back to empty where the chains
            // claimed (every cell after a cancelled row pass), before the
            // next window's pass; after the leg's last window the leg end
            // does it
            if (w + 1 < b.windows) {
                for (int w2 = lw * gridDim.x + blockIdx.x; w2 < total_chains; w2 += nwarps) {
                    const int r = find_rep(b.chain_base, R, w2);
                    if (!rep_on(b, r)) continue;
                    const Dev &s = warp_dev(my_dev, my_rep, b.reps, r);
                    if (!(s.rp_ok && s.rp[RP_BAD + par] == 0) ||
                        __ldcg(s.rp + RP_ABORT + par) != 0)
                        continue;
                    row_reset_chain<C>(s, w2 - b.chain_base[r]);
                }
                for (int r = 0; r < R; ++r) {
                    if (!rep_on(b, r)) continue;
                    const Dev &s = b.reps[r];
                    if (s.rp_ok && s.rp[RP_BAD + par] == 0 && __ldcg(s.rp + RP_ABORT + par) != 0)
                        clear_row_claims(s, gt, nthreads);
                }
            }
            // repair rounds
            for (int round = 1;; ++round) {
                if (!(round == 1 && uf_early)) {
                    for (int r = blockIdx.x; r < R; r += gridDim.x) uf_replica(r, round);
                    // the last block to finish its union-finds takes the
                    // prefix: no grid barrier between
                    if (last_block()) comp_prefix();
                    if (!grid_barrier(b, &sflag)) return;
                }
                const int ncomp = b.g[G_ANY];
                if (ncomp == 0) break;
                for (;;) {
                    int q = 0;
                    if (lane == 0) q = atomicAdd(b.g + G_WORK, 1);
                    q = __shfl_sync(FULL, q, 0);
                    if (q >= ncomp) break;
                    const int r = find_rep(b.comp_base, R, q);
                    const Dev &s = warp_dev(my_dev, my_rep, b.reps, r);
                    repair_component<C>(s, q - b.comp_base[r], round, window_start(s, w),
                                        window_end(s, w));
                }
                if (!grid_barrier(b, &sflag)) return;
                // no component met another chain: the window is repaired
                int aborted = 0;
                for (int r = threadIdx.x; r < R; r += blockDim.x)
                    if (rep_on(b, r) && b.reps[r].ctl[CTL_NABORT] != 0) aborted = 1;
                if (!__syncthreads_or(aborted)) break;
            }
            mark(PH_REPAIR);
        }
        // leg end: liftings and the log, then per-replica totals and budgets;
        // a warp whose chains share a replica adds their liftings at once.
        // The claim words are cleared for the next leg here, off the next
        // leg's begin (whose few dependent loads per chain would queue
        // behind the stores)
        // (and the row pass's claim arrays of the last window: where the
        // chains claimed, or every cell after a cancelled row pass)
        const int pl = (p0 + b.windows - 1) & 1;
        for (int r = 0; r < R; ++r) {
            if (!rep_on(b, r)) continue;
            const Dev &s = b.reps[r];
            clear_claims(s, gt, nthreads);
            if (s.rp_ok && s.rp[RP_BAD + pl] == 0 && __ldcg(s.rp + RP_ABORT + pl) != 0)
                clear_row_claims(s, gt, nthreads);
        }
        // one chain per warp (the next leg's start clears the chain's records
        // lane-parallel); with one system the block adds its liftings at once
        if (threadIdx.x == 0) blk_lifts = 0ull;
        __syncthreads();
        for (int w2 = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; w2 < total_chains;
             w2 += nwarps) {
            const int r = find_rep(b.chain_base, R, w2);
            if (!rep_on(b, r)) continue;
            const Dev &s = warp_dev(my_dev, my_rep, b.reps, r);
            const int c = w2 - b.chain_base[r];
            if (s.rp_ok && s.rp[RP_BAD + pl] == 0 && __ldcg(s.rp + RP_ABORT + pl) == 0)
                row_reset_chain<C>(s, c);
            int32_t nl = 0;
            if (lane == 0)
                nl = leg_end_chain(s, c, (int32_t)(b.ctl[r].leg_index0 + b.ctl[r].legs), false);
            __syncwarp();
            bool ok = true;
            if (next_leg_at_end(b, r, leg)) {
                ok = leg_begin_chain_warp(s, c, lane);
                if (lane == 0 && s.rp_ok && skip_of(s, s.aloc[c]) != RP_SKIP_ALL)
                    atomicAdd(s.rp + RP_BAD + (((leg + 1) * b.windows) & 1), 1);
            } else if (lane == 0) {
                ok = s.cid[s.aloc[c]] == s.ci[c];
            }
            if (lane == 0) {
                // chain table against the cells (must hold: every chain has
                // stalled on the disk its slot names)
                if (!ok && atomicAdd(&b.ctl[r].incons, 1) == 0) {
                    b.ctl[r].bad_where = leg * 65536 + (b.windows - 1) * 16 + 15;
                    b.ctl[r].bad_chain = c;
                }
                if (nl) {
                    if (R == 1)
                        atomicAdd(&blk_lifts, (unsigned long long)nl);
                    else
                        atomicAdd(s.lc + LC_LIFTS, (unsigned long long)nl);
                }
            }
        }
        __syncthreads();
        if (R == 1 && threadIdx.x == 0 && blk_lifts)
            atomicAdd(b.reps[0].lc + LC_LIFTS, blk_lifts);
        // the last block to finish takes the totals (one grid barrier for
        // both)
        const bool totals_here = last_block();
        for (int r = threadIdx.x; totals_here && r < R; r += blockDim.x) {
            // (the control block, the counters and the pointers read into
            // registers first: one round trip, not one per field)
            RepCtl *const cp = b.ctl + r;
            RepCtl c = *cp;
            if (!(c.live && !c.done)) continue;
            unsigned long long *const lcp = b.reps[r].lc;
            int32_t *const rpp = b.reps[r].rp;
            unsigned long long lc[LC_N];
#pragma unroll
            for (int q = 0; q < LC_N; ++q) lc[q] = __ldcg(lcp + q);
            const int flag = lc[LC_BLOCKED] != 0ull || lc[LC_WEAK] != 0ull;
            if (c.flags && c.legs < c.flags_cap) c.flags[c.legs] = (uint8_t)flag;
            c.lifts += (int64_t)lc[LC_LIFTS];
            c.p1_lifts += (int64_t)lc[LC_P1LIFTS];
            if (flag) c.repair_lifts += (int64_t)lc[LC_LIFTS];
            c.legs += 1;
            c.conflict_legs += flag;
            c.repaired += (int64_t)lc[LC_REPAIRED];
            c.continued += (int64_t)lc[LC_CONTINUED];
            c.row_windows += (int64_t)lc[LC_ROWWIN];
            c.blocked += (int64_t)lc[LC_BLOCKED];
            c.cwindows += (int64_t)lc[LC_CWINDOWS];
            c.horizon += (int64_t)lc[LC_HORIZON];
            c.order_err += (int64_t)lc[LC_ORDER];
            if (lc[LC_ERR_CAP] || lc[LC_ERR_REC]) c.err = 1;
            if (c.err || (c.budget > 0 && c.lifts >= c.budget)) c.done = 1;
            const bool next_begun = c.budget == 0 && leg + 1 < b.max_legs;
            *cp = c;
            // per-leg counters back to zero for the next leg; the row-pass
            // counters of the leg's last window (a next leg begun above has
            // counted into the other parity)
#pragma unroll
            for (int q = 0; q < LC_N; ++q) lcp[q] = 0ull;
            if (next_begun) {
                rpp[RP_BAD + pl] = 0;
                rpp[RP_ABORT + pl] = 0;
            } else {
                rpp[RP_BAD] = 0;
                rpp[RP_BAD + 1] = 0;
                rpp[RP_ABORT] = 0;
                rpp[RP_ABORT + 1] = 0;
            }
            if (!c.done) atomicAdd(b.g + G_REMAIN0 + (leg & 1), 1);
        }
        if (!grid_barrier(b, &sflag)) return;
        mark(PH_END);
        if (b.g[G_REMAIN0 + (leg & 1)] == 0) break;
    }
    // the replicas whose internal checks recorded a failure (Dev::dbg[0]),
    // for the host, which reads the details of those only
    if (blockIdx.x == 0)
        for (int r = threadIdx.x; r < R; r += blockDim.x)
            if (b.reps[r].dbg && __ldcg(b.reps[r].dbg) != 0.0) b.ctl[r].dbg = 1;
}

}  // namespace

// ------------------------------------------------------------------ host

// ------------------------------------------------ device memory cache

namespace {
struct CudaBackend {
    int alloc(void **p, size_t bytes) {
        const cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) (void)cudaGetLastError();
        return (int)e;
    }
    void free(void *p) { cudaFree(p); }
};
constexpr int DM_MAX_DEVICES = 64;
constexpr size_t DM_DEFAULT_LIMIT = (size_t)4 << 30;  // cached bytes per device
std::mutex g_dm_mu;
BlockCache<CudaBackend> *g_dm[DM_MAX_DEVICES];
size_t g_dm_limit = DM_DEFAULT_LIMIT;

// The cache of device dev (created on first use, never destroyed: its blocks
// would outlive the CUDA runtime at process exit).
BlockCache<CudaBackend> *dm_cache(int dev) {
    if (dev < 0 || dev >= DM_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lock(g_dm_mu);
    if (!g_dm[dev]) g_dm[dev] = new BlockCache<CudaBackend>(g_dm_limit);
    return g_dm[dev];
}
}  // namespace

int dm_alloc(void **p, size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = -1;
    }
    BlockCache<CudaBackend> *c = dm_cache(dev);
    if (!c) return CudaBackend().alloc(p, bytes);
    return c->acquire(p, bytes);
}

void dm_free(void *p) {
    if (!p) return;
    // the block goes back to the cache of the device that holds it
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaPointerGetAttributes(&a, p) == cudaSuccess)
        dev = a.device;
    else
        (void)cudaGetLastError();
    BlockCache<CudaBackend> *c = dm_cache(dev);
    if (c)
        c->release(p);
    else
        cudaFree(p);
}

extern "C" int ecmc_set_cache_limit(int64_t bytes) {
    if (bytes < 0) return ECMC_EINVAL;
    std::lock_guard<std::mutex> lock(g_dm_mu);
    g_dm_limit = (size_t)bytes;
    for (auto *c : g_dm)
        if (c) c->set_limit(g_dm_limit);
    return ECMC_OK;
}

extern "C" int ecmc_cache_info(int64_t *cached_bytes, int64_t *in_use_bytes, int64_t *hits,
                               int64_t *misses) {
    DevCacheInfo t = {0, 0, 0, 0};
    {
        std::lock_guard<std::mutex> lock(g_dm_mu);
        for (auto *c : g_dm) {
            if (!c) continue;
            const DevCacheInfo i = c->info();
            t.cached_bytes += i.cached_bytes;
            t.in_use_bytes += i.in_use_bytes;
            t.hits += i.hits;
            t.misses += i.misses;
        }
    }
    if (cached_bytes) *cached_bytes = t.cached_bytes;
    if (in_use_bytes) *in_use_bytes = t.in_use_bytes;
    if (hits) *hits = t.hits;
    if (misses) *misses = t.misses;
    return ECMC_OK;
}

// Launch scratch of the persistent kernel (reps, barrier, counters).
struct Runner {
    int cap = 0;
    // one device block: [reps | chain_base | comp_base | ctl | bar | g | phase]
    // (256-byte aligned parts), uploaded whole before a launch and read back
    // from ctl on after it, through `host` (one copy each way)
    unsigned char *block = nullptr;
    size_t off_base = 0, off_comp = 0, off_ctl = 0, off_bar = 0, off_g = 0, off_phase = 0,
           total = 0;
    std::vector<unsigned char> host;
    Dev *d_reps = nullptr;
    RepCtl *d_ctl = nullptr;
    int32_t *d_chain_base = nullptr, *d_comp_base = nullptr;
    unsigned int *d_bar = nullptr;
    int32_t *d_g = nullptr;
    unsigned long long *d_phase = nullptr;
    int grid4 = 0, grid8 = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    GBatchScratch *gscratch = nullptr;  // batches of constraint-graph contexts
};

static void runner_free(Runner &rn) {
    graph_batch_free(rn.gscratch);
    rn.gscratch = nullptr;
    dm_free(rn.block);
    if (rn.ev0) cudaEventDestroy(rn.ev0);
    if (rn.ev1) cudaEventDestroy(rn.ev1);
    rn = Runner();
}

struct ecmc_ctx {
    ecmc_params p;
    Dev s;
    Runner run;
    uint8_t *d_flags = nullptr;
    int32_t flags_cap = 0;
    int C = 4;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<void *> allocs;
    // device arrays requested by dalloc, placed in one allocation by pool_commit
    std::vector<std::pair<void **, size_t>> pending;
    // scratch of ecmc_positions, kept for the next call
    double *exp_x = nullptr, *exp_y = nullptr, *exp_t = nullptr;
    int32_t *exp_a = nullptr;
    ecmc_profile_t prof = {};
    int n_sm = 1;
    int64_t legs_total = 0;
    int64_t lifts_total = 0;
    int64_t conflict_legs = 0;
    int64_t repaired = 0;
    int64_t continued = 0;
    int64_t restarts = 0;
    int64_t row_windows = 0;
    int64_t blocked = 0;
    int64_t cwindows = 0;
    int64_t device_bytes = 0;  // device memory held by the context
    unsigned long long wait_ns = BARRIER_TIMEOUT_NS;  // bound on device waits
    int64_t horizon = 0;
    int64_t order_err = 0;
    int64_t inconsistent = 0;
    double device_ms = 0.0;
    bool log_overflow = false;
    int32_t direction = 0;  // 0: +x; 1: +y (the context is stored transposed)
    GraphCtx *graph = nullptr;  // ECMC_GRAPH: the constraint-graph path holds the state
};

static std::string g_create_err;

static int fail(ecmc_ctx *ctx, int code, const std::string &msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_err = msg;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, ECMC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
static int dalloc(ecmc_ctx *ctx, T **ptr, size_t count) {
    *ptr = nullptr;
    ctx->pending.emplace_back((void **)ptr, std::max<size_t>(count, 1) * sizeof(T));
    return 0;
}

// One device block (from the device memory cache) for every array requested
// since the last commit, each starting on a 256-byte boundary.
static int pool_commit(ecmc_ctx *ctx) {
    size_t total = 0;
    for (auto &r : ctx->pending) total += (r.second + 255) & ~(size_t)255;
    void *base = nullptr;
    if (total) {
        const int e = dm_alloc(&base, total);
        if (e != 0) {
            ctx->pending.clear();
            return fail(ctx, ECMC_ENOMEM,
                        std::string("cudaMalloc: ") + cudaGetErrorString((cudaError_t)e));
        }
        ctx->allocs.push_back(base);
        ctx->device_bytes += (int64_t)total;
    }
    size_t off = 0;
    for (auto &r : ctx->pending) {
        *r.first = (char *)base + off;
        off += (r.second + 255) & ~(size_t)255;
    }
    ctx->pending.clear();
    return 0;
}

// FP32 image of the stop rule thr(m) = ((m a) - fx) - d > RN(cur + eps):
// thr_f = ((m af - fxf) - df) and lim_f = trunc(cur) + epsf, with af, df, epsf
// the FP32 roundings, fxf = trunc(fx). Each of the four FP32 roundings and
// the two truncations errs by at most 2^-23 of a term of magnitude at most
// m a + a + d + cur + eps <= L + a + d + ell + eps (m < nc, |fx| <= a,
// cur <= ell), so |(thr_f - lim_f) - (thr - lim)| < 2^-22 (L + a + d + ell +
// eps) (the FP64 roundings are 2^29 times smaller). stop_e is 4 times that.
static void set_stop_image(Dev &s) {
    s.af = (float)s.a;
    s.df = (float)s.d;
    s.epsf = (float)s.eps;
    s.stop_e = (float)std::ldexp(s.L + s.a + s.d + s.ell + s.eps + 1.0, -20);
}

// Exact tables of the cell map cell_coord(v) = min(nc - 1, trunc(RN(v inv_a))):
// colx[c] = RN(c a) and xbound[c] = the least double v >= 0 with
// cell_coord(v) >= c, found from c a by steps of one ulp (the map is
// monotone). Host and device multiply alike (IEEE binary64, round to nearest).
static void cell_tables(const Dev &s, std::vector<double> &colx,
                        std::vector<unsigned long long> &xb) {
    const int nc = s.nc;
    colx.resize(nc);
    xb.assign((size_t)nc + 1, 0ull);
    auto at_least = [&](double v, int c) { return v * s.inv_a >= (double)c; };
    for (int c = 0; c < nc; ++c) colx[c] = (double)c * s.a;
    for (int c = 1; c < nc; ++c) {
        double v = (double)c * s.a;
        while (v > 0.0 && at_least(std::nextafter(v, 0.0), c)) v = std::nextafter(v, 0.0);
        while (!at_least(v, c)) v = std::nextafter(v, INFINITY);
        unsigned long long b;
        memcpy(&b, &v, 8);
        xb[c] = b;
    }
    const double inf = INFINITY;
    memcpy(&xb[nc], &inf, 8);
}

static int pick_cells(const ecmc_params *p, int *nc_out, int *C_out) {
    const double d = p->d, L = p->box;
    int nc = p->cells_per_side;
    if (nc == 0) {
        nc = (int)(L / (d * (1.0 + std::ldexp(1.0, -20))));
        while (nc > 3 && !(L / nc >= d * (1.0 + std::ldexp(1.0, -20)))) --nc;
    }
    if (nc < 3) return -1;
    const double a = L / nc;
    if (!(a >= d * (1.0 + std::ldexp(1.0, -20)))) return -1;
    // At most 4 centres at mutual distance >= d fit in a cell with a < sqrt(2) d
    // (one per quadrant); at most 6 for a < 1.664 d (a 3 x 2 split).
    int C;
    if (a < std::sqrt(2.0) * d * (1.0 - 1e-9))
        C = 4;
    else if (a < 1.664 * d)
        C = 8;
    else
        return -1;
    *nc_out = nc;
    *C_out = C;
    return 0;
}

// ECMC_GRAPH: the state lives in the constraint-graph path (graph.cu).
static int create_graph(ecmc_ctx *ctx, int nc, const double *x, const double *y,
                        const int32_t *active) {
    const ecmc_params *p = &ctx->p;
    const bool dev_in = (p->flags & ECMC_INPUT_DEVICE) != 0;
    int rc = 0;
    const size_t n = (size_t)p->n, k = (size_t)p->n_chains;
    // one scratch allocation: the uploaded inputs, the ids seen, two counters
    const size_t off_y = n * 8, off_a = 2 * n * 8, off_seen = (off_a + k * 4 + 15) & ~(size_t)15;
    const size_t off_bad = (off_seen + n * 4 + 15) & ~(size_t)15;
    char *scratch = nullptr;
    if (dm_alloc_t(&scratch, off_bad + 16) != 0) {
        g_create_err = "cudaMalloc failed (inputs)";
        return ECMC_ENOMEM;
    }
    double *dx = (double *)scratch, *dy = (double *)(scratch + off_y);
    int32_t *da = (int32_t *)(scratch + off_a);
    uint32_t *seen = (uint32_t *)(scratch + off_seen);
    unsigned long long *bad = (unsigned long long *)(scratch + off_bad);
    const double *sx = x, *sy = y;
    const int32_t *sa = active;
    auto release = [&]() {
        // (copies or the check may still read the scratch after a failure)
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) (void)cudaGetLastError();
        dm_free(scratch);
    };
    if (!dev_in) {
        if (cudaMemcpyAsync(dx, x, n * 8, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(dy, y, n * 8, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(da, active, k * 4, cudaMemcpyHostToDevice, ctx->stream) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            release();
            g_create_err = "input upload";
            return ECMC_ECUDA;
        }
        sx = dx;
        sy = dy;
        sa = da;
    }
    {
        unsigned long long hb[2] = {0ull, 0ull};
        cudaError_t e = cudaMemsetAsync(seen, 0, off_bad + 16 - off_seen, ctx->stream);
        if (e == cudaSuccess) {
            launch_check(sx, sy, sa, (int64_t)n, (int)k, p->box, seen, bad, bad + 1, ctx->stream);
            e = cudaMemcpyAsync(hb, bad, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            release();
            g_create_err = "input check";
            return ECMC_ECUDA;
        }
        if (hb[0] || hb[1]) {
            release();
            g_create_err = hb[0] ? "coordinate outside [0, L)"
                                 : "active ids must be distinct and in [0, n)";
            return ECMC_EINVAL;
        }
    }
    std::string err;
    rc = graph_create(p, nc, sx, sy, sa, ctx->stream, &ctx->graph, err);
    cudaStreamSynchronize(ctx->stream);
    release();
    if (rc) g_create_err = err;
    return rc;
}


// Device arrays of a cell-scan context, set up but not allocated yet: the
// scalar description in ctx->s and one request per array in ctx->pending
// (ecmc_create commits them; ecmc_context_bytes only adds them up).
struct CreateArrays {
    double *colx = nullptr;
    unsigned long long *xbound = nullptr;
    uint32_t *loc_of = nullptr;
    double *dx = nullptr, *dy = nullptr;
    int32_t *dact = nullptr;
};

static int plan_cell_context(ecmc_ctx *ctx, const ecmc_params *p, int nc, int C,
                             CreateArrays *out) {
    Dev &s = ctx->s;
    memset(&s, 0, sizeof s);
    s.n = p->n;
    s.nc = nc;
    s.k = p->n_chains;
    s.cap = p->undo_cap > 0 ? p->undo_cap : 1024;
    s.windows = p->windows > 0 ? p->windows : 1;
    s.L = p->box;
    s.d = p->d;
    s.d2 = p->d * p->d;
    s.ell = p->ell;
    s.a = p->box / (double)nc;
    s.inv_a = (double)nc / p->box;
    s.far = s.L - 3.0 * s.a;
    s.eps = std::ldexp(p->box, -30);
    set_stop_image(s);
    s.log_on = (p->flags & ECMC_LOG_LIFTINGS) ? 1 : 0;
    s.log_cap = s.log_on ? (p->log_cap > 0 ? p->log_cap : ((int64_t)1 << 22)) : 0;
    const size_t ncell = (size_t)nc * nc;
    const size_t nslot = ncell * C;
    const size_t n = (size_t)p->n, k = (size_t)p->n_chains;
    int rc = 0;
    auto chk = [&](int r) {
        if (r && !rc) rc = r;
    };
    chk(dalloc(ctx, &s.cx, nslot));
    chk(dalloc(ctx, &s.cy, nslot));
    chk(dalloc(ctx, &s.ct, nslot));
    chk(dalloc(ctx, &s.cid, nslot));
    chk(dalloc(ctx, &s.cown, nslot));
    chk(dalloc(ctx, &s.cskp, nslot));
    chk(dalloc(ctx, &s.rband, 2 * (size_t)nc));
    chk(dalloc(ctx, &out->colx, (size_t)nc));
    chk(dalloc(ctx, &out->xbound, (size_t)nc + 1));
    chk(dalloc(ctx, &s.claim, ncell));
    // the row pass needs a window of 32 / C columns well inside the ring and
    // a leg shorter than L - 3a (no disk behind the active disk in reach)
    s.rp_ok = (!(p->flags & ECMC_NO_ROWPASS) && nc >= 4 * (32 / C) && p->ell < s.far &&
               p->n_chains < (1 << 29)) ? 1 : 0;
    if (s.rp_ok) {
        chk(dalloc(ctx, &s.ckey, ncell));
        chk(dalloc(ctx, &s.camin, ncell));
        chk(dalloc(ctx, &s.camax, ncell));
    }
    chk(dalloc(ctx, &s.rp, RP_N));
    chk(dalloc(ctx, &s.rp_n, k));
    chk(dalloc(ctx, &s.rp_front, k));
    chk(dalloc(ctx, &s.rp_end, k));
    chk(dalloc(ctx, &s.rp_partner, k));
    chk(dalloc(ctx, &s.rp_aloc, k));
    chk(dalloc(ctx, &s.rp_start, k));
    chk(dalloc(ctx, &s.rp_ci, k));
    chk(dalloc(ctx, &s.rp_tc, k));
    chk(dalloc(ctx, &s.rp_D, k));
    chk(dalloc(ctx, &s.aloc0, k));
    chk(dalloc(ctx, &s.aloc, k));
    chk(dalloc(ctx, &s.ci, k));
    chk(dalloc(ctx, &s.D, k));
    chk(dalloc(ctx, &s.tc, k));
    chk(dalloc(ctx, &s.status, k));
    chk(dalloc(ctx, &s.partner, k));
    chk(dalloc(ctx, &s.nrec, k));
    chk(dalloc(ctx, &s.nlift, k));
    chk(dalloc(ctx, &s.rec, k * (size_t)s.cap));
    chk(dalloc(ctx, &s.ev_T, k));
    chk(dalloc(ctx, &s.ev_tau, k));
    chk(dalloc(ctx, &s.ev_xj, k));
    chk(dalloc(ctx, &s.ev_yj, k));
    chk(dalloc(ctx, &s.ev_tj, k));
    chk(dalloc(ctx, &s.vt, k));
    chk(dalloc(ctx, &s.uf, k));
    chk(dalloc(ctx, &s.fin, k));
    chk(dalloc(ctx, &s.comp_of, k));
    chk(dalloc(ctx, &s.abort_to, k));
    chk(dalloc(ctx, &s.comp_cnt, k));
    chk(dalloc(ctx, &s.comp_off, k + 1));
    chk(dalloc(ctx, &s.comp_root, k));
    chk(dalloc(ctx, &s.comp_mem, k));
    chk(dalloc(ctx, &s.blist, k));
    chk(dalloc(ctx, &s.pcnt, k));
    chk(dalloc(ctx, &s.ctl, CTL_N));
    chk(dalloc(ctx, &s.dbg, 16));
    chk(dalloc(ctx, &s.ev_j, k));
    chk(dalloc(ctx, &s.ev_jloc, k));
    chk(dalloc(ctx, &s.ev_lift, k));
    chk(dalloc(ctx, &s.ev_cx, k));
    chk(dalloc(ctx, &s.ev_cy, k));
    chk(dalloc(ctx, &s.ev_mlast, k));
    chk(dalloc(ctx, &s.lc, LC_N));
    chk(dalloc(ctx, &s.tc_cnt, TC_N));
    if (s.log_on) chk(dalloc(ctx, &s.log, (size_t)s.log_cap));
    chk(dalloc(ctx, &out->loc_of, n));
    if (!(p->flags & ECMC_INPUT_DEVICE)) {
        chk(dalloc(ctx, &out->dx, n));
        chk(dalloc(ctx, &out->dy, n));
        chk(dalloc(ctx, &out->dact, k));
    }
    return rc;
}

extern "C" int ecmc_context_bytes(const ecmc_params *p, int64_t *bytes) {
    if (!p || !bytes) return ECMC_EINVAL;
    if (p->n < 3 || p->n > (int64_t)0x3FFFFFFF || p->n_chains < 1 || p->n_chains > p->n)
        return ECMC_EINVAL;
    if (p->undo_cap < 0 || p->undo_cap >= (1 << 24) || !(p->box > 0.0) || !(p->d > 0.0) ||
        !(p->ell > 0.0))
        return ECMC_EINVAL;
    int nc = 0, C = 4;
    if (pick_cells(p, &nc, &C)) return ECMC_EINVAL;
    ecmc_ctx *ctx = new (std::nothrow) ecmc_ctx();
    if (!ctx) return ECMC_ENOMEM;
    CreateArrays arr;
    int64_t graph_bytes = 0;
    if (p->flags & ECMC_GRAPH) {
        // the graph context's own arrays; the cell-scan arrays are not made
        graph_bytes = graph_plan_bytes(p, nc);
        if (graph_bytes < 0) {
            delete ctx;
            return ECMC_EINVAL;
        }
    } else {
        plan_cell_context(ctx, p, nc, C, &arr);
    }
    // the export scratch of ecmc_positions (allocated by its first call)
    dalloc(ctx, &ctx->exp_x, (size_t)p->n);
    dalloc(ctx, &ctx->exp_y, (size_t)p->n);
    dalloc(ctx, &ctx->exp_t, (size_t)p->n);
    dalloc(ctx, &ctx->exp_a, (size_t)p->n_chains);
    int64_t total = graph_bytes;
    for (auto &r : ctx->pending) total += (int64_t)((r.second + 255) & ~(size_t)255);
    ctx->pending.clear();
    ctx->exp_x = nullptr;
    ctx->exp_y = nullptr;
    ctx->exp_t = nullptr;
    ctx->exp_a = nullptr;
    delete ctx;
    *bytes = total;
    return ECMC_OK;
}

extern "C" int ecmc_create(const ecmc_params *p, const double *x, const double *y,
                           const int32_t *active, void *stream, ecmc_ctx **out) {
    ecmc_ctx *ctx = nullptr;
    if (!p || !x || !y || !active || !out) return fail(nullptr, ECMC_EINVAL, "null argument");
    *out = nullptr;
    if (p->n < 3 || p->n > (int64_t)0x3FFFFFFF) return fail(nullptr, ECMC_EINVAL, "n out of range");
    if (p->n_chains < 1 || p->n_chains > p->n) return fail(nullptr, ECMC_EINVAL, "n_chains out of range");
    if (p->windows < 0 || p->windows > 4096) return fail(nullptr, ECMC_EINVAL, "windows out of range");
    if (p->undo_cap < 0 || p->undo_cap >= (1 << 24))
        return fail(nullptr, ECMC_EINVAL, "undo_cap out of range (0 .. 2^24 - 1)");
    if (!(p->d > 0.0) || !(p->ell > 0.0) || !(p->box > 0.0) || !std::isfinite(p->box) ||
        !std::isfinite(p->ell))
        return fail(nullptr, ECMC_EINVAL, "d, ell and box must be positive and finite");
    int nc = 0, C = 4;
    if (pick_cells(p, &nc, &C))
        return fail(nullptr, ECMC_EINVAL, "cell geometry: need nc >= 3 and d < L/nc < 1.664 d");
    if ((int64_t)nc * nc * C > (int64_t)0xFFFFFFF0)
        return fail(nullptr, ECMC_EINVAL, "too many cells");

    ctx = new (std::nothrow) ecmc_ctx();
    if (!ctx) return fail(nullptr, ECMC_ENOMEM, "host allocation");
    ctx->p = *p;
    ctx->stream = (cudaStream_t)stream;
    ctx->C = C;
    if ((p->flags & ECMC_RESTART) && (!(p->flags & ECMC_GRAPH) || p->windows > 1)) {
        delete ctx;
        return fail(nullptr, ECMC_EINVAL, "ECMC_RESTART needs ECMC_GRAPH and one claim window");
    }
    if (p->flags & ECMC_GRAPH) {
        memset(&ctx->s, 0, sizeof ctx->s);
        ctx->s.n = p->n;
        ctx->s.k = p->n_chains;
        const int rc = create_graph(ctx, nc, x, y, active);
        if (rc) {
            ecmc_destroy(ctx);
            return rc;
        }
        *out = ctx;
        return ECMC_OK;
    }
    Dev &s = ctx->s;
    CreateArrays arr;
    int rc = plan_cell_context(ctx, p, nc, C, &arr);
    auto chk = [&](int r) {
        if (r && !rc) rc = r;
    };
    const size_t ncell = (size_t)nc * nc;
    const size_t nslot = ncell * C;
    const size_t n = (size_t)p->n, k = (size_t)p->n_chains;
    const bool dev_in = (p->flags & ECMC_INPUT_DEVICE) != 0;
    chk(pool_commit(ctx));
    if (rc) {
        g_create_err = ctx->err;
        ecmc_destroy(ctx);
        return rc;
    }
    double *const dx = arr.dx, *const dy = arr.dy, *const d_colx = arr.colx;
    int32_t *const dact = arr.dact;
    uint32_t *const loc_of = arr.loc_of;
    unsigned long long *const d_xbound = arr.xbound;
    cudaStream_t st = ctx->stream;
    const double *sx = x, *sy = y;
    const int32_t *sa = active;
    if (!dev_in) {
        CU(cudaMemcpyAsync(dx, x, n * 8, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(dy, y, n * 8, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(dact, active, k * 4, cudaMemcpyHostToDevice, st));
        sx = dx;
        sy = dy;
        sa = dact;
    }
    CU(cudaMemsetAsync(s.cid, 0xFF, nslot * sizeof(uint32_t), st));
    CU(cudaMemsetAsync(s.claim, 0, ncell * sizeof(uint32_t), st));
    CU(cudaMemsetAsync(s.pcnt, 0, (size_t)s.k * sizeof(int32_t), st));
    CU(cudaMemsetAsync(s.rp, 0, RP_N * sizeof(int32_t), st));
    if (s.rp_ok) {
        CU(cudaMemsetAsync(s.ckey, 0xFF, ncell * sizeof(unsigned long long), st));
        CU(cudaMemsetAsync(s.camin, 0xFF, ncell * sizeof(uint32_t), st));
        CU(cudaMemsetAsync(s.camax, 0, ncell * sizeof(uint32_t), st));
    }
    CU(cudaMemsetAsync(s.lc, 0, LC_N * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(s.tc_cnt, 0, TC_N * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(s.nrec, 0, k * sizeof(int32_t), st));
    CU(cudaMemsetAsync(s.dbg, 0, 16 * sizeof(double), st));
    {
        std::vector<double> colx;
        std::vector<unsigned long long> xb;
        cell_tables(s, colx, xb);
        CU(cudaMemcpyAsync(d_colx, colx.data(), colx.size() * 8, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(d_xbound, xb.data(), xb.size() * 8, cudaMemcpyHostToDevice, st));
        // (pageable sources: the copies are done when the calls return)
        s.colx = d_colx;
        s.xbound = d_xbound;
    }
    // the inputs are checked on the device: the active ids here (loc_of holds
    // the ids seen until k_fill writes the slots into it), the coordinates by
    // k_place; nothing below indexes by an active id before k_init_chains,
    // which does nothing if an id failed
    CU(cudaMemsetAsync(loc_of, 0, n * sizeof(uint32_t), st));
    launch_check(nullptr, nullptr, sa, (int64_t)n, (int)k, s.L, loc_of, s.lc + LC_BADXY,
                 s.lc + LC_BADID, st);
    if (C == 4)
        launch_cells<4>(s, sx, sy, loc_of, s.lc + LC_BADXY, st);
    else
        launch_cells<8>(s, sx, sy, loc_of, s.lc + LC_BADXY, st);
    launch_skip(s, C, st);
    k_init_chains<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(s, sa, loc_of);
    CU(cudaGetLastError());
    {
        int dev = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev));
    }
    unsigned long long h_lc[LC_N];
    CU(cudaMemcpyAsync(h_lc, s.lc, LC_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h_lc[LC_BADXY] || h_lc[LC_BADID]) {
        g_create_err = h_lc[LC_BADXY] ? "coordinate outside [0, L)"
                                      : "active ids must be distinct and in [0, n)";
        ecmc_destroy(ctx);
        return ECMC_EINVAL;
    }
    if (h_lc[LC_ERR_CAP]) {
        g_create_err = "more disks in a cell than it has slots (overlapping input?)";
        ecmc_destroy(ctx);
        return ECMC_ECAPACITY;
    }
    CU(cudaMemsetAsync(s.lc, 0, LC_N * sizeof(unsigned long long), st));
    *out = ctx;
    return ECMC_OK;
}

// Grids of the persistent launch on the current device (SMs x resident
// blocks, for 4 and 8 slots per cell): queried once per device.
static bool run_grids(int *grid4, int *grid8) {
    static std::mutex mu;
    static int g4[DM_MAX_DEVICES], g8[DM_MAX_DEVICES];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lock(mu);
    const bool cached = dev >= 0 && dev < DM_MAX_DEVICES && g4[dev] > 0;
    if (!cached) {
        int n_sm = 1, b4 = 0, b8 = 0, coop = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, k_run<4>, RUN_THREADS,
                                                          UF_SMEM_BYTES) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b8, k_run<8>, RUN_THREADS,
                                                          UF_SMEM_BYTES) != cudaSuccess ||
            !coop || b4 < 1 || b8 < 1) {
            (void)cudaGetLastError();
            return false;
        }
        if (dev >= 0 && dev < DM_MAX_DEVICES) {
            g4[dev] = n_sm * b4;
            g8[dev] = n_sm * b8;
        }
        *grid4 = n_sm * b4;
        *grid8 = n_sm * b8;
        return true;
    }
    *grid4 = g4[dev];
    *grid8 = g8[dev];
    return true;
}

static int runner_reserve(Runner &rn, int R, std::string &err) {
    if (rn.cap >= R && rn.d_reps) return 0;
    runner_free(rn);
    const int cap = std::max(R, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    (void)take(cap * sizeof(Dev));
    rn.off_base = take((cap + 1) * sizeof(int32_t));
    rn.off_comp = take((cap + 1) * sizeof(int32_t));
    rn.off_ctl = take(cap * sizeof(RepCtl));
    rn.off_bar = take(2 * sizeof(unsigned int));
    rn.off_g = take(G_N * sizeof(int32_t));
    rn.off_phase = take(PH_N * sizeof(unsigned long long));
    rn.total = off;
    rn.host.assign(rn.total, 0);
    if (dm_alloc_t(&rn.block, rn.total) != 0 ||
        cudaEventCreate(&rn.ev0) != cudaSuccess || cudaEventCreate(&rn.ev1) != cudaSuccess) {
        (void)cudaGetLastError();
        runner_free(rn);
        err = "runner allocation failed";
        return ECMC_ENOMEM;
    }
    int grid4 = 0, grid8 = 0;
    if (!run_grids(&grid4, &grid8)) {
        runner_free(rn);
        err = "cooperative launch unavailable";
        return ECMC_ECUDA;
    }
    rn.grid4 = grid4;
    rn.grid8 = grid8;
    rn.d_reps = (Dev *)rn.block;
    rn.d_chain_base = (int32_t *)(rn.block + rn.off_base);
    rn.d_comp_base = (int32_t *)(rn.block + rn.off_comp);
    rn.d_ctl = (RepCtl *)(rn.block + rn.off_ctl);
    rn.d_bar = (unsigned int *)(rn.block + rn.off_bar);
    rn.d_g = (int32_t *)(rn.block + rn.off_g);
    rn.d_phase = (unsigned long long *)(rn.block + rn.off_phase);
    rn.cap = cap;
    return 0;
}

// Runs up to max_legs legs of every context in one persistent launch on
// `st`; per-context totals are folded into each context's host counters.
static int runner_run(Runner &rn, cudaStream_t st, ecmc_ctx *const *ctxs, int R, int32_t max_legs,
                      const uint64_t *budgets, int64_t *lifts_out, int32_t *legs_out,
                      std::string &err, double *ms_out) {
    if (R < 1 || max_legs < 0) {
        err = "bad batch size or leg count";
        return ECMC_EINVAL;
    }
    for (int r = 0; r < R; ++r)
        if (!ctxs[r] || (ctxs[r]->graph != nullptr) != (ctxs[0]->graph != nullptr)) {
            err = "a batch holds either constraint-graph contexts or cell-scan contexts";
            return ECMC_EINVAL;
        }
    if (ctxs[0]->graph) {
        // constraint-graph contexts: their own persistent kernel over all of them
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < r; ++q)
                if (ctxs[q] == ctxs[r]) {
                    err = "a context appears twice in a batch";
                    return ECMC_EINVAL;
                }
        std::vector<GraphCtx *> gs(R);
        std::vector<GraphTotals> tots(R);
        for (int r = 0; r < R; ++r) gs[r] = ctxs[r]->graph;
        double ms = 0.0;
        const int grc = graph_batch_run(&rn.gscratch, gs.data(), R, max_legs, budgets, st,
                                        tots.data(), legs_out, &ms, err);
        if (ms_out) *ms_out = ms;
        for (int r = 0; r < R; ++r) {
            ecmc_ctx *c = ctxs[r];
            const GraphTotals &t = tots[r];
            c->legs_total += t.legs;
            c->lifts_total += t.lifts;
            c->conflict_legs += t.conflict_legs;
            c->repaired += t.repaired;
            c->continued += t.continued;
            c->blocked += t.blocked;
            c->cwindows += t.cwindows;
            c->horizon += t.horizon;
            c->order_err += t.order_err;
            c->prof.pass1_launches += t.legs;
            c->prof.other_launches += t.legs;
            c->prof.repair_launches += t.conflict_legs;
            c->prof.pass1_liftings += t.p1_lifts;
            c->prof.repair_liftings += t.repair_lifts;
            if (R == 1) {
                c->device_ms += t.ms;
                c->prof.pass1_ms += t.pass1_ms;
                c->prof.repair_ms += t.repair_ms;
                c->prof.other_ms += t.other_ms;
            }
            if (lifts_out) lifts_out[r] = t.lifts;
        }
        return grc;
    }
    const int C = ctxs[0]->C;
    const int W = ctxs[0]->s.windows;
    for (int r = 0; r < R; ++r) {
        if (!ctxs[r] || ctxs[r]->C != C || ctxs[r]->s.windows != W) {
            err = "all contexts of a batch need the same cell slots (cell size) and windows";
            return ECMC_EINVAL;
        }
        for (int q = 0; q < r; ++q)
            if (ctxs[q] == ctxs[r]) {
                err = "a context appears twice in a batch";
                return ECMC_EINVAL;
            }
    }
    int rc = runner_reserve(rn, R, err);
    if (rc) return rc;
    if (max_legs == 0) return 0;
    std::vector<Dev> reps(R);
    std::vector<RepCtl> ctl(R);
    std::vector<int32_t> base(R + 1, 0);
    for (int r = 0; r < R; ++r) {
        ecmc_ctx *c = ctxs[r];
        if (c->stream != st && cudaStreamSynchronize(c->stream) != cudaSuccess) {
            err = "context stream";
            return ECMC_ECUDA;
        }
        if (c->flags_cap < max_legs) {
            dm_free(c->d_flags);
            c->d_flags = nullptr;
            c->flags_cap = 0;
            if (dm_alloc_t(&c->d_flags, (size_t)max_legs) != 0) {
                err = "flags allocation";
                return ECMC_ENOMEM;
            }
            c->flags_cap = max_legs;
        }
        reps[r] = c->s;
        memset(&ctl[r], 0, sizeof(RepCtl));
        ctl[r].budget = budgets ? (int64_t)budgets[r] : 0;
        ctl[r].leg_index0 = c->legs_total;
        ctl[r].flags = c->d_flags;
        ctl[r].flags_cap = c->flags_cap;
        ctl[r].live = 1;
        base[r + 1] = base[r] + c->s.k;
    }
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && !rc) {
            (void)cudaGetLastError();
            err = std::string(what) + ": " + cudaGetErrorString(e);
            rc = ECMC_ECUDA;
        }
    };
    // the tables and zeroed barrier, counters and phase times: one copy
    unsigned char *h = rn.host.data();
    memcpy(h, reps.data(), R * sizeof(Dev));
    memcpy(h + rn.off_base, base.data(), (R + 1) * sizeof(int32_t));
    memcpy(h + rn.off_ctl, ctl.data(), R * sizeof(RepCtl));
    memset(h + rn.off_bar, 0, rn.total - rn.off_bar);
    cu(cudaMemcpyAsync(rn.block, h, rn.total, cudaMemcpyHostToDevice, st), "tables");
    if (rc) return rc;
    Batch b;
    b.reps = rn.d_reps;
    b.ctl = rn.d_ctl;
    b.chain_base = rn.d_chain_base;
    b.comp_base = rn.d_comp_base;
    b.bar = rn.d_bar;
    b.g = rn.d_g;
    b.phase_ns = rn.d_phase;
    b.R = R;
    b.max_legs = max_legs;
    b.windows = W;
    b.pad = 0;
    b.wait_ns = BARRIER_TIMEOUT_NS;
    for (int r = 0; r < R; ++r) b.wait_ns = std::min(b.wait_ns, ctxs[r]->wait_ns);
    void *args[] = {&b};
    cu(cudaEventRecord(rn.ev0, st), "event");
    if (C == 4)
        cu(cudaLaunchCooperativeKernel((void *)k_run<4>, rn.grid4, RUN_THREADS, args, UF_SMEM_BYTES,
                                       st), "launch");
    else
        cu(cudaLaunchCooperativeKernel((void *)k_run<8>, rn.grid8, RUN_THREADS, args, UF_SMEM_BYTES,
                                       st), "launch");
    cu(cudaEventRecord(rn.ev1, st), "event");
    int32_t g[G_N];
    unsigned long long ph[PH_N];
    // control blocks, counters and phase times back: one copy
    cu(cudaMemcpyAsync(h + rn.off_ctl, rn.block + rn.off_ctl, rn.total - rn.off_ctl,
                       cudaMemcpyDeviceToHost, st), "tables");
    cu(cudaStreamSynchronize(st), "run");
    if (rc) return rc;
    memcpy(ctl.data(), h + rn.off_ctl, R * sizeof(RepCtl));
    memcpy(g, h + rn.off_g, sizeof g);
    memcpy(ph, h + rn.off_phase, sizeof ph);
    float ms = 0.f;
    cu(cudaEventElapsedTime(&ms, rn.ev0, rn.ev1), "elapsed");
    if (ms_out) *ms_out = ms;
    bool cap_err = false, incons_err = false;
    std::string incons_msg;
    for (int r = 0; r < R; ++r) {
        ecmc_ctx *c = ctxs[r];
        const RepCtl &q = ctl[r];
        c->legs_total += q.legs;
        c->lifts_total += q.lifts;
        c->conflict_legs += q.conflict_legs;
        c->repaired += q.repaired;
        c->continued += q.continued;
        c->row_windows += q.row_windows;
        c->blocked += q.blocked;
        c->cwindows += q.cwindows;
        c->horizon += q.horizon;
        c->order_err += q.order_err;
        c->prof.pass1_launches += q.legs;
        c->prof.other_launches += q.legs;
        c->prof.repair_launches += q.conflict_legs;
        c->prof.pass1_liftings += q.p1_lifts;
        c->prof.repair_liftings += q.repair_lifts;
        if (R == 1) {
            c->prof.pass1_ms += ph[PH_PASS1] * 1e-6;
            c->prof.repair_ms += ph[PH_REPAIR] * 1e-6;
            c->prof.other_ms += (ph[PH_BEGIN] + ph[PH_END]) * 1e-6;
            c->device_ms += ms;
        }
        if (lifts_out) lifts_out[r] = q.lifts;
        if (legs_out) legs_out[r] = (int32_t)q.legs;
        if (q.err) cap_err = true;
        if (q.incons) {
            c->inconsistent += q.incons;
            if (!incons_err) {
                char buf[160];
                snprintf(buf, sizeof buf,
                         "chain table check failed %d times; first: leg %d window %d phase %d chain %d",
                         q.incons, q.bad_where / 65536, (q.bad_where % 65536) / 16,
                         q.bad_where % 16, q.bad_chain);
                incons_msg = buf;
            }
            incons_err = true;
        }
    }
    if (g[G_ERR] == ECMC_ETIMEOUT) {
        err = "a grid barrier wait passed its time limit";
        return ECMC_ETIMEOUT;
    }
    if (cap_err) {
        err = "cell slots, undo records or repair rounds overflowed";
        return ECMC_ECAPACITY;
    }
    for (int r = 0; r < R; ++r) {
        double dg[7];
        // (the launch flagged the replicas whose internal checks recorded
        // something; only those are read)
        if (ctl[r].dbg && ctxs[r]->s.dbg &&
            cudaMemcpy(dg, ctxs[r]->s.dbg, sizeof dg, cudaMemcpyDeviceToHost) == cudaSuccess &&
            dg[0] != 0.0) {
            char buf[240];
            snprintf(buf, sizeof buf, "internal check %g failed: %.17g %.17g %.17g %.17g %.17g %.17g",
                     dg[0], dg[1], dg[2], dg[3], dg[4], dg[5], dg[6]);
            err = buf;
            return ECMC_ECUDA;
        }
    }
    if (incons_err) {
        err = incons_msg;
        return ECMC_ECUDA;
    }
    return 0;
}

extern "C" int ecmc_run_to_breakpoint(ecmc_ctx *ctx, int32_t n_legs, uint64_t event_budget,
                                      uint8_t *leg_flags_out, int32_t *legs_done) {
    if (!ctx) return ECMC_EINVAL;
    if (n_legs < 0) return fail(ctx, ECMC_EINVAL, "n_legs < 0");
    if (legs_done) *legs_done = 0;
    if (n_legs == 0) return ECMC_OK;
    if (ctx->graph) {
        GraphTotals t;
        std::string err;
        int32_t legs = 0;
        const int rc = graph_run(ctx->graph, n_legs, event_budget, leg_flags_out, &legs, &t, err);
        if (legs_done) *legs_done = legs;
        ctx->legs_total += t.legs;
        ctx->lifts_total += t.lifts;
        ctx->conflict_legs += t.conflict_legs;
        ctx->repaired += t.repaired;
        ctx->continued += t.continued;
        ctx->restarts += t.restarts;
        ctx->blocked += t.blocked;
        ctx->cwindows += t.cwindows;
        ctx->horizon += t.horizon;
        ctx->order_err += t.order_err;
        ctx->device_ms += t.ms;
        ctx->prof.pass1_launches += t.legs;
        ctx->prof.other_launches += t.legs;
        ctx->prof.repair_launches += t.conflict_legs;
        ctx->prof.pass1_liftings += t.p1_lifts;
        ctx->prof.repair_liftings += t.repair_lifts;
        ctx->prof.pass1_ms += t.pass1_ms;
        ctx->prof.repair_ms += t.repair_ms;
        ctx->prof.other_ms += t.other_ms;
        if (rc) return fail(ctx, rc, err);
        return ECMC_OK;
    }
    ecmc_ctx *one[1] = {ctx};
    int32_t legs = 0;
    std::string err;
    const int rc = runner_run(ctx->run, ctx->stream, one, 1, n_legs, &event_budget, nullptr, &legs,
                              err, nullptr);
    if (legs_done) *legs_done = legs;
    if (leg_flags_out && legs > 0) {
        CU(cudaMemcpyAsync(leg_flags_out, ctx->d_flags, (size_t)legs, cudaMemcpyDeviceToHost,
                           ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    if (rc) return fail(ctx, rc, err);
    return ECMC_OK;
}

struct ecmc_batch {
    Runner run;
    cudaStream_t stream = nullptr;
    std::string err;
    double device_ms = 0.0;
};

extern "C" int ecmc_batch_create(void *stream, ecmc_batch **out) {
    if (!out) return ECMC_EINVAL;
    ecmc_batch *b = new (std::nothrow) ecmc_batch();
    if (!b) return ECMC_ENOMEM;
    b->stream = (cudaStream_t)stream;
    *out = b;
    return ECMC_OK;
}

extern "C" int ecmc_batch_run(ecmc_batch *b, ecmc_ctx *const *ctxs, int32_t n_ctx,
                              int32_t max_legs, const uint64_t *budgets, int64_t *liftings_out,
                              int32_t *legs_out, double *device_ms_out) {
    if (!b || !ctxs || n_ctx < 1) return ECMC_EINVAL;
    double ms = 0.0;
    const int rc = runner_run(b->run, b->stream, ctxs, n_ctx, max_legs, budgets, liftings_out,
                              legs_out, b->err, &ms);
    b->device_ms += ms;
    if (device_ms_out) *device_ms_out = ms;
    return rc;
}

extern "C" const char *ecmc_batch_last_error(const ecmc_batch *b) {
    return b ? b->err.c_str() : "";
}

extern "C" void ecmc_batch_destroy(ecmc_batch *b) {
    if (!b) return;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) (void)cudaGetLastError();
    runner_free(b->run);
    delete b;
}

extern "C" int ecmc_positions(ecmc_ctx *ctx, double *x, double *y, double *t, int32_t *active) {
    if (!ctx) return ECMC_EINVAL;
    Dev &s = ctx->s;
    cudaStream_t st = ctx->stream;
    const size_t n = (size_t)s.n;
    const size_t nslot = (size_t)s.nc * s.nc * ctx->C;
    // device scratch, allocated at the first call and kept by the context
    if (!ctx->exp_x) {
        dalloc(ctx, &ctx->exp_x, n);
        dalloc(ctx, &ctx->exp_y, n);
        dalloc(ctx, &ctx->exp_t, n);
        dalloc(ctx, &ctx->exp_a, (size_t)s.k);
        const int rc = pool_commit(ctx);
        if (rc) return rc;
    }
    double *dx = x ? ctx->exp_x : nullptr, *dy = y ? ctx->exp_y : nullptr;
    double *dt = t ? ctx->exp_t : nullptr;
    int32_t *da = active ? ctx->exp_a : nullptr;
    if (ctx->graph) {
        double *ex = ctx->direction ? dy : dx, *ey = ctx->direction ? dx : dy;
        if (graph_export(ctx->graph, ex, ey, dt, da) != 0)
            return fail(ctx, ECMC_ECUDA, "positions (graph)");
    } else if (x || y || t) {
        // in a transposed context the stored x is the caller's y
        double *ex = ctx->direction ? dy : dx, *ey = ctx->direction ? dx : dy;
        if (ctx->C == 4)
            k_export<4><<<(unsigned)((nslot + 255) / 256), 256, 0, st>>>(s, ex, ey, dt);
        else
            k_export<8><<<(unsigned)((nslot + 255) / 256), 256, 0, st>>>(s, ex, ey, dt);
    }
    if (active && !ctx->graph)
        k_export_active<<<(unsigned)((s.k + 127) / 128), 128, 0, st>>>(s, da);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && x) e = cudaMemcpyAsync(x, dx, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && y) e = cudaMemcpyAsync(y, dy, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && t) e = cudaMemcpyAsync(t, dt, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && active)
        e = cudaMemcpyAsync(active, da, (size_t)s.k * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ctx, ECMC_ECUDA, std::string("positions: ") + cudaGetErrorString(e));
    return ECMC_OK;
}

extern "C" int ecmc_set_direction(ecmc_ctx *ctx, int32_t direction) {
    if (!ctx) return ECMC_EINVAL;
    if (direction != 0 && direction != 1) return fail(ctx, ECMC_EINVAL, "direction must be 0 (+x) or 1 (+y)");
    if (direction == ctx->direction) return ECMC_OK;
    if (ctx->graph) {
        std::string err;
        const int rc = graph_transpose(ctx->graph, err);
        if (rc) return fail(ctx, rc, "set_direction: " + err);
        ctx->direction = direction;
        return ECMC_OK;
    }
    Dev &s = ctx->s;
    cudaStream_t st = ctx->stream;
    const int64_t ncell = (int64_t)s.nc * s.nc;
    if (ctx->C == 4) {
        k_transpose<4><<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(s);
        k_transpose_chains<4><<<(unsigned)((s.k + 127) / 128), 128, 0, st>>>(s);
    } else {
        k_transpose<8><<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(s);
        k_transpose_chains<8><<<(unsigned)((s.k + 127) / 128), 128, 0, st>>>(s);
    }
    launch_skip(s, ctx->C, st);  // rows are the old columns
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ctx, ECMC_ECUDA, std::string("set_direction: ") + cudaGetErrorString(e));
    ctx->direction = direction;
    return ECMC_OK;
}

extern "C" int ecmc_set_wait_limit(ecmc_ctx *ctx, uint64_t ns) {
    if (!ctx) return ECMC_EINVAL;
    if (ns == 0 || ns > BARRIER_TIMEOUT_NS) return fail(ctx, ECMC_EINVAL, "wait limit out of range");
    ctx->wait_ns = ns;
    return ECMC_OK;
}

extern "C" int ecmc_stats(ecmc_ctx *ctx, ecmc_stats_t *out) {
    if (!ctx || !out) return ECMC_EINVAL;
    out->liftings = ctx->lifts_total;
    out->legs = ctx->legs_total;
    out->conflict_legs = ctx->conflict_legs;
    out->repaired_chains = ctx->repaired;
    out->continued_chains = ctx->continued;
    out->restarts = ctx->restarts;
    out->row_windows = ctx->row_windows;
    out->blocked_chains = ctx->blocked;
    out->conflict_windows = ctx->cwindows;
    out->device_bytes = (ctx->graph ? graph_device_bytes(ctx->graph) : 0) + ctx->device_bytes;
    out->horizon_asserts = ctx->horizon;
    out->order_errors = ctx->order_err;
    out->device_ms = ctx->device_ms;
    return ECMC_OK;
}

extern "C" int ecmc_profile(ecmc_ctx *ctx, ecmc_profile_t *out) {
    if (!ctx || !out) return ECMC_EINVAL;
    *out = ctx->prof;
    return ECMC_OK;
}

extern "C" int ecmc_graph_arrows(ecmc_ctx *ctx, int32_t *a, double *b) {
    if (!ctx) return ECMC_EINVAL;
    if (!ctx->graph) return fail(ctx, ECMC_EINVAL, "not a constraint-graph context");
    std::string err;
    const int rc = graph_arrows(ctx->graph, a, b, err);
    return rc ? fail(ctx, rc, err) : ECMC_OK;
}

extern "C" int ecmc_liftings(ecmc_ctx *ctx, ecmc_lift_t *buf, int64_t cap, int64_t *n_out) {
    if (!ctx || !n_out) return ECMC_EINVAL;
    if (ctx->graph) {
        std::string err;
        const int rc = graph_liftings(ctx->graph, buf, cap, n_out, err);
        return rc ? fail(ctx, rc, err) : ECMC_OK;
    }
    Dev &s = ctx->s;
    if (!s.log_on) return fail(ctx, ECMC_EINVAL, "lifting log not enabled");
    unsigned long long n = 0;
    CU(cudaMemcpyAsync(&n, s.tc_cnt + TC_LOG_N, sizeof n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *n_out = (int64_t)n;
    if ((int64_t)n > s.log_cap) return fail(ctx, ECMC_ECAPACITY, "lifting log overflowed log_cap");
    std::vector<ecmc_lift_t> all((size_t)n);
    if (n) {
        CU(cudaMemcpyAsync(all.data(), s.log, n * sizeof(ecmc_lift_t), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    // chains append their records concurrently; order leg by leg, chain by chain
    std::stable_sort(all.begin(), all.end(), [](const ecmc_lift_t &a, const ecmc_lift_t &b) {
        return a.leg != b.leg ? a.leg < b.leg : a.c < b.c;
    });
    if (buf && cap > 0)
        memcpy(buf, all.data(), (size_t)std::min<int64_t>(cap, (int64_t)n) * sizeof(ecmc_lift_t));
    return ECMC_OK;
}

extern "C" void ecmc_destroy(ecmc_ctx *ctx) {
    if (!ctx) return;
    // (every call on the context has synchronised its stream before
    // returning; this one makes sure before its blocks go to the cache)
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) (void)cudaGetLastError();
    graph_destroy(ctx->graph);
    runner_free(ctx->run);
    dm_free(ctx->d_flags);
    for (void *p : ctx->allocs) dm_free(p);
    delete ctx;
}

extern "C" const char *ecmc_last_error(const ecmc_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

// ------------------------------------------ one leg without any allocation
//
// For callers that cannot allocate device memory: code that runs while a
// framework owns the whole device heap through its own caching allocator
// (a cudaMalloc would fail or fragment that pool), real-time loops that must
// not pay allocation latency, and plug-ins that are only handed pointers.
// All working memory of the leg comes from one file-scope device array of
// fixed size; the caller passes only inputs and outputs.

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)ECMC_NOALLOC_SCRATCH_MIB << 20;
constexpr int NOALLOC_CAP = ECMC_NOALLOC_RECORDS;  // event records per chain per leg
constexpr int NOALLOC_MAX_DEVICES = 64;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array for the current device, looked up once.
static int noalloc_scratch(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return ECMC_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return ECMC_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = (unsigned char *)g_noalloc_ptr[dev];
    return ECMC_OK;
}

// Lays the arrays of Dev out in [base, base + bytes); with base == nullptr
// only the size is computed.
struct Carve {
    unsigned char *base;
    size_t off;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += std::max<size_t>(count, 1) * sizeof(T);
        return p;
    }
};

static size_t noalloc_layout(Dev &s, unsigned char *base, size_t nslot, size_t ncell, size_t n,
                             size_t k, uint32_t **loc_of) {
    Carve cv{base, 0};
    s.cx = cv.take<double>(nslot);
    s.cy = cv.take<double>(nslot);
    s.ct = cv.take<double>(nslot);
    s.cid = cv.take<uint32_t>(nslot);
    s.cown = cv.take<uint32_t>(nslot);
    s.claim = cv.take<uint32_t>(ncell);
    *loc_of = cv.take<uint32_t>(n);
    s.aloc0 = cv.take<uint32_t>(k);
    s.aloc = cv.take<uint32_t>(k);
    s.ci = cv.take<uint32_t>(k);
    s.D = cv.take<double>(k);
    s.tc = cv.take<double>(k);
    s.status = cv.take<int32_t>(k);
    s.partner = cv.take<int32_t>(k);
    s.nrec = cv.take<int32_t>(k);
    s.nlift = cv.take<int32_t>(k);
    s.ev_T = cv.take<double>(k);
    s.ev_tau = cv.take<double>(k);
    s.ev_xj = cv.take<double>(k);
    s.ev_yj = cv.take<double>(k);
    s.ev_tj = cv.take<double>(k);
    s.ev_j = cv.take<uint32_t>(k);
    s.ev_jloc = cv.take<uint32_t>(k);
    s.ev_lift = cv.take<int32_t>(k);
    s.ev_cx = cv.take<int32_t>(k);
    s.ev_cy = cv.take<int32_t>(k);
    s.ev_mlast = cv.take<int32_t>(k);
    s.vt = cv.take<double>(k);
    s.uf = cv.take<int32_t>(k);
    s.fin = cv.take<int32_t>(k);
    s.comp_of = cv.take<int32_t>(k);
    s.abort_to = cv.take<int32_t>(k);
    s.comp_cnt = cv.take<int32_t>(k);
    s.comp_off = cv.take<int32_t>(k + 1);
    s.comp_root = cv.take<int32_t>(k);
    s.comp_mem = cv.take<int32_t>(k);
    s.blist = cv.take<int32_t>(k);
    s.pcnt = cv.take<int32_t>(k);
    s.ctl = cv.take<int32_t>(CTL_N);
    s.lc = cv.take<unsigned long long>(LC_N);
    s.tc_cnt = cv.take<unsigned long long>(TC_N);
    s.rec = cv.take<Rec>(k * (size_t)s.cap);
    return cv.off;
}

#define CUN(call)                                   \
    do {                                            \
        if ((call) != cudaSuccess) {                \
            (void)cudaGetLastError();               \
            return ECMC_ECUDA;                      \
        }                                           \
    } while (0)

template <int C>
static int noalloc_leg(Dev &s, cudaStream_t st, int n_sm, uint8_t *flag, int64_t *lifts) {
    unsigned long long lc[LC_N];
    int32_t ctl[CTL_N];
    const unsigned kb = (unsigned)((s.k + 127) / 128);
    CUN(cudaMemsetAsync(s.lc, 0, LC_N * sizeof(unsigned long long), st));
    CUN(cudaMemsetAsync(s.pcnt, 0, (size_t)s.k * sizeof(int32_t), st));
    k_leg_begin<<<kb, 128, 0, st>>>(s);
    CUN(cudaMemsetAsync(s.claim, 0, (size_t)s.nc * s.nc * sizeof(uint32_t), st));
    k_pass1<C><<<(unsigned)((s.k + 3) / 4), 128, 0, st>>>(s);
    CUN(cudaGetLastError());
    CUN(cudaMemcpyAsync(lc, s.lc, sizeof lc, cudaMemcpyDeviceToHost, st));
    CUN(cudaStreamSynchronize(st));
    if (lc[LC_ERR_CAP] || lc[LC_ERR_REC]) return ECMC_ECAPACITY;
    const bool conflict = lc[LC_BLOCKED] != 0;
    if (conflict) {
        for (int round = 1;; ++round) {
            if (round > 255) return ECMC_ECAPACITY;
            k_uf<<<1, 1024, 0, st>>>(s, round == 1);
            k_repair<C><<<(unsigned)(n_sm * 4), 128, 0, st>>>(s, round);
            CUN(cudaGetLastError());
            CUN(cudaMemcpyAsync(ctl, s.ctl, sizeof ctl, cudaMemcpyDeviceToHost, st));
            CUN(cudaStreamSynchronize(st));
            if (ctl[CTL_NABORT] == 0) break;
        }
    }
    k_leg_end<<<kb, 128, 0, st>>>(s, 0);
    CUN(cudaGetLastError());
    CUN(cudaMemcpyAsync(lc, s.lc, sizeof lc, cudaMemcpyDeviceToHost, st));
    CUN(cudaStreamSynchronize(st));
    if (lc[LC_ERR_CAP] || lc[LC_ERR_REC]) return ECMC_ECAPACITY;
    if (flag) *flag = (conflict || lc[LC_WEAK] != 0) ? 1 : 0;
    if (lifts) *lifts = (int64_t)lc[LC_LIFTS];
    return ECMC_OK;
}

template <int C>
static int noalloc_run(Dev &s, uint32_t *loc_of, double *x, const double *y, int32_t *active,
                       double *t_out, cudaStream_t st, int n_sm, uint8_t *flag, int64_t *lifts) {
    const size_t nslot = (size_t)s.nc * s.nc * C;
    unsigned long long lc[LC_N];
    CUN(cudaMemsetAsync(s.cid, 0xFF, nslot * sizeof(uint32_t), st));
    launch_check(x, y, active, s.n, s.k, s.L, loc_of, s.lc + LC_ERR_CAP, s.lc + LC_ERR_CAP, st);
    CUN(cudaGetLastError());
    CUN(cudaMemcpyAsync(lc, s.lc, sizeof lc, cudaMemcpyDeviceToHost, st));
    CUN(cudaStreamSynchronize(st));
    if (lc[LC_ERR_CAP]) return ECMC_EINVAL;
    launch_cells<C>(s, x, y, loc_of, nullptr, st);
    k_init_chains<<<(unsigned)((s.k + 255) / 256), 256, 0, st>>>(s, active, loc_of);
    CUN(cudaGetLastError());
    CUN(cudaMemcpyAsync(lc, s.lc, sizeof lc, cudaMemcpyDeviceToHost, st));
    CUN(cudaStreamSynchronize(st));
    if (lc[LC_ERR_CAP]) return ECMC_ECAPACITY;  // more disks in a cell than slots
    const int rc = noalloc_leg<C>(s, st, n_sm, flag, lifts);
    if (rc) return rc;
    k_export<C><<<(unsigned)((nslot + 255) / 256), 256, 0, st>>>(s, x, nullptr, t_out);
    k_export_active<<<(unsigned)((s.k + 127) / 128), 128, 0, st>>>(s, active);
    CUN(cudaGetLastError());
    CUN(cudaStreamSynchronize(st));
    return ECMC_OK;
}

}  // namespace

extern "C" int ecmc_leg_noalloc(int64_t n, double box, double d, double ell, int32_t n_chains,
                                int32_t cells_per_side, double *x, const double *y,
                                int32_t *active, double *t_out, void *stream, uint8_t *flag_out,
                                int64_t *lifts_out) {
    if (!x || !y || !active) return ECMC_EINVAL;
    if (n < 3 || n > (int64_t)0x3FFFFFFF || n_chains < 1 || n_chains > n) return ECMC_EINVAL;
    if (!(d > 0.0) || !(ell > 0.0) || !(box > 0.0) || !std::isfinite(box) || !std::isfinite(ell))
        return ECMC_EINVAL;
    ecmc_params p;
    memset(&p, 0, sizeof p);
    p.n = n;
    p.box = box;
    p.d = d;
    p.ell = ell;
    p.n_chains = n_chains;
    p.cells_per_side = cells_per_side;
    int nc = 0, C = 4;
    if (pick_cells(&p, &nc, &C)) return ECMC_EINVAL;
    Dev s;
    memset(&s, 0, sizeof s);
    s.n = n;
    s.nc = nc;
    s.k = n_chains;
    s.cap = NOALLOC_CAP;
    s.windows = 1;
    s.L = box;
    s.d = d;
    s.d2 = d * d;
    s.ell = ell;
    s.a = box / (double)nc;
    s.inv_a = (double)nc / box;
    s.far = s.L - 3.0 * s.a;
    s.eps = std::ldexp(box, -30);
    set_stop_image(s);
    const size_t ncell = (size_t)nc * nc, nslot = ncell * C;
    uint32_t *loc_of = nullptr;
    // sizes beyond the fixed scratch array are rejected before any device work
    if (noalloc_layout(s, nullptr, nslot, ncell, (size_t)n, (size_t)n_chains, &loc_of) >
        NOALLOC_SCRATCH_BYTES)
        return ECMC_EINVAL;
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    const size_t used = noalloc_layout(s, base, nslot, ncell, (size_t)n, (size_t)n_chains, &loc_of);
    int dev = 0, n_sm = 1;
    CUN(cudaGetDevice(&dev));
    CUN(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: start from zero
    CUN(cudaMemsetAsync(base, 0, used, st));
    rc = C == 4 ? noalloc_run<4>(s, loc_of, x, y, active, t_out, st, n_sm, flag_out, lifts_out)
                : noalloc_run<8>(s, loc_of, x, y, active, t_out, st, n_sm, flag_out, lifts_out);
    return rc;
}
