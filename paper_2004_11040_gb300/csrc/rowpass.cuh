// rowpass.cuh -- the parallel pass of a claim window for chains that move
// along one cell row ("row pass"); included by ecmc.cu inside its unnamed
// namespace, after the cell-scan step it shares the stop rule and tables with.
//
// When the rows above and below a disk's cell row hold no disk within d of it
// in y (its skip bits are 3, see k_skip), a chain there never leaves the row
// during the leg: a lifting goes to a disk within d in y, which lies in the
// same row. For a window in which every running chain of a system is in that
// case, the pass runs as below instead of pass1_chain. Results are unchanged
// (Alg. 2, bit for bit); only the way the pass is computed differs.
//
//  * Speculation. Every chain runs alone from the window-start state -- the
//    isolated run of the conflict flag (the oracle's definition) -- and no
//    chain writes a cell during the pass. A warp holds G = 32 / C consecutive
//    columns of its row in registers, one slot per lane, and slides forward.
//  * Few FP64 instructions per step. On this GPU every FP64 warp instruction
//    occupies its SM sub-partition's FP64 unit for ~64 cycles, whatever its
//    lane mask, so the step is arranged around their count:
//      - when the window slides, b = sqrt(d^2 - dy^2) of every disk towards
//        the next disk of the window in x order is computed for all lanes by
//        one instruction sequence; that next disk is the predicted target;
//      - per step, dx for every lane, then ONE subtraction that gives the
//        predicted target's tau = dx - b and every other lane's lower bound
//        dx - d (tau >= dx - d because b <= d, and RN is monotone). The
//        prediction stands when every other scanned candidate's bound lies
//        above tau (for a stall: at or above D); otherwise the step is
//        evaluated exactly, lane by lane, as scan_step does (rp_exact);
//      - t_i + tau, x_i + tau, D - tau and the next disk's offset in its cell
//        are one lane-parallel addition.
//  * Claims. Every scanned cell gets fire-and-forget atomics: the least claim
//    key (strong before weak, then earlier local time, then lower chain), and
//    the least and largest claiming chain. After a grid barrier each chain
//    (row_resolve_chain) finds the first cell of its row that another chain
//    holds, publishes its events before the step that first scanned that
//    cell, and is blocked there with the holder as partner; every scanned
//    cell gets its holder's claim word. The state the repair starts from is
//    then of the kind pass1_chain leaves: each chain's applied events lie in
//    cells that no other chain's applied events touch (a run of Alg. 3
//    without violations so far), and Lemma 2's continuation and the
//    global-order replay finish the window as before.
//  * Flag. Two chains' isolated claim sets meet iff some cell has two
//    claiming chains: exactly the oracle's flag.
//  * Anything outside the common case -- a scan wider than the window, a next
//    active disk whose rows are in reach, an advance close to a lap, a full
//    record log or cell -- cancels the speculative pass of that system for
//    the window (nothing was written) and pass1_chain runs in its place.

constexpr unsigned long long RP_WEAK = 1ull << 63;
constexpr uint32_t RP_SKIP_ALL = 3u;
enum { RP_END_STALL = 0, RP_END_PAUSE = 1, RP_END_NONSTATIC = 2 };
// Dev::rp: [RP_BAD + parity] chains whose rows are in reach, [RP_ABORT +
// parity] row pass cancelled, for windows of even and odd parity
enum { RP_BAD = 0, RP_ABORT = 2, RP_N = 4 };

// Claim key of chain c reading (strong) or covering (weak) a cell at local
// time ti >= 0 (its FP32 image rounded toward zero: monotone in ti), m
// columns ahead of its active disk's column. The least key holds the cell:
// strong before weak, then the earlier scan, then the nearer column (at equal
// times, as at every chain's first step, a chain keeps the column of its own
// active disk), then the lower chain. Any such order is exact; this one makes
// the chain that reaches a cell later in its own time the one that waits.
constexpr int RP_KEY_MBITS = 3;
__device__ __forceinline__ unsigned long long rp_key(int c, double ti, int m, bool weak) {
    const unsigned tb = (unsigned)__float_as_int(d2f_trunc(ti));
    const unsigned mm = m < (1 << RP_KEY_MBITS) - 1 ? (unsigned)m : (1u << RP_KEY_MBITS) - 1u;
    return (weak ? RP_WEAK : 0ull) | ((unsigned long long)tb << 32) |
           ((unsigned long long)mm << 29) | (unsigned long long)c;
}
constexpr unsigned long long RP_KEY_CHAIN = (1ull << 29) - 1ull;

// One lane of the window: one slot of one column of the chain's row.
struct RowLane {
    uint32_t id, own, skp;
    double x, y, t;
    int nx;                       // lane of the next disk in x order, -1 none
    int bok;                      // b is that of a disk within d in y
    double b;                     // sqrt(d^2 - dy^2) towards lane nx
    unsigned long long xlo, xhi;  // xbound of the lane's column and of the next
    double colx;                  // left edge of the lane's column
};

// Uniform state of the chain run by the warp.
struct RowChain {
    int c, row, u0;  // chain, cell row, column of the active disk at the window start
    int wbase;       // column offset (from u0) of window position 0
    int gbase;       // lane group holding window position 0
    int li;          // lane of the active disk
    uint32_t i, iskp;
    double xi, yi, ti, D, fx;
    int front;       // last column offset claimed in this window, -1 none
    int32_t nrec0, n;  // first record of the window, records written
    int lifts;
};

template <int C>
__device__ __forceinline__ int rp_pos(const RowChain &ch) {
    constexpr int G = 32 / C;
    return (((threadIdx.x & 31) / C) - ch.gbase) & (G - 1);
}

// Slot held by lane l (uniform arithmetic: no shuffle).
template <int C>
__device__ __forceinline__ uint32_t rp_loc_of(const Dev &s, const RowChain &ch, int l) {
    constexpr int G = 32 / C;
    int col = ch.u0 + ch.wbase + (((l / C) - ch.gbase) & (G - 1));
    if (col >= s.nc) col -= s.nc;
    return ((uint32_t)ch.row * (uint32_t)s.nc + (uint32_t)col) * C + (uint32_t)(l % C);
}

// Loads this lane's slot (window position pos) from the window-start state.
template <int C>
__device__ void rp_load(const Dev &s, const RowChain &ch, RowLane &w, int pos) {
    int col = ch.u0 + ch.wbase + pos;
    if (col >= s.nc) col -= s.nc;
    const uint32_t loc = ((uint32_t)ch.row * (uint32_t)s.nc + (uint32_t)col) * C +
                         (threadIdx.x & 31) % C;
    w.id = s.cid[loc];
    w.x = s.cx[loc];
    w.y = s.cy[loc];
    w.t = s.ct[loc];
    w.own = s.cown[loc];
    w.skp = s.cskp[loc];
    w.xlo = s.xbound[col];
    w.xhi = s.xbound[col + 1];
    w.colx = s.colx[col];
}

// L2 prefetch of the G columns that follow the window (offsets off .. off +
// G - 1 from the chain's start column): the slot arrays of the active row,
// the row-skip bits and the column bounds that the next slide loads. After
// the L2 flush between launches every window's first touch would otherwise
// wait on DRAM (a chain moves forward, never back, within a leg).
template <int C>
__device__ __forceinline__ void rp_prefetch(const Dev &s, const RowChain &ch, int off) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31;
    const int e = lane >> 2, f = lane & 3;  // column off + e (e < 8), field pair f
    if (e >= G) return;
    int col = ch.u0 + off + e;
    while (col >= s.nc) col -= s.nc;
    const uint32_t loc = ((uint32_t)ch.row * (uint32_t)s.nc + (uint32_t)col) * C;
    const void *p0, *p1;
    if (f == 0) {
        p0 = s.cx + loc;
        p1 = s.cy + loc;
    } else if (f == 1) {
        p0 = s.ct + loc;
        p1 = s.cid + loc;
    } else if (f == 2) {
        p0 = s.cown + loc;
        p1 = s.cskp + loc;
    } else {
        p0 = s.xbound + col;
        p1 = s.colx + col;
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p0));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p1));
}

// Next disk in x order within the window (by window position, then x) and b
// towards it, for every lane: one FP64 instruction sequence for all lanes.
template <int C>
__device__ void rp_links(const Dev &s, const RowChain &ch, RowLane &w, int *nx_raw = nullptr,
                         int *rank_out = nullptr) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31, g = lane / C, q = lane % C;
    const int v = (g - ch.gbase) & (G - 1);
    const bool occ = w.id != EMPTY;
    // x >= 0 and below 2^11 L-units: the bits order like the values and fit
    // below the position field
    const unsigned long long key =
        occ ? (((unsigned long long)v << 59) | (dbits(w.x) >> 5)) : ~0ull;
    int rank = 0;
#pragma unroll
    for (int q2 = 0; q2 < C; ++q2) {
        const unsigned long long k2 = shfl_u64(key, g * C + q2);
        rank += (k2 < key) || (k2 == key && q2 < q);
    }
    const unsigned gm = ((1u << C) - 1u) << (g * C);
    unsigned succ = 0u;  // lanes holding the rank after mine
#pragma unroll
    for (int r = 1; r < C; ++r) {
        const unsigned rm = __ballot_sync(FULL, occ && rank == r);
        if (rank + 1 == r) succ = rm;
    }
    const unsigned first = __ballot_sync(FULL, occ && rank == 0);
    int nx = -1;
    if (occ) {
        if (succ & gm) {
            nx = __ffs(succ & gm) - 1;
        } else {
            for (int dv = 1; v + dv < G; ++dv) {
                const int g2 = (ch.gbase + v + dv) & (G - 1);
                const unsigned m2 = first & (((1u << C) - 1u) << (g2 * C));
                if (m2) {
                    nx = __ffs(m2) - 1;
                    break;
                }
            }
        }
    }
    w.nx = nx;
    if (nx_raw) *nx_raw = nx;
    if (rank_out) *rank_out = rank;
    // the same operations as scan_step: |y_target - y_active| (one row: no
    // periodic image), then sqrt(d^2 - ay^2)
    const double yn = __shfl_sync(FULL, w.y, nx >= 0 ? nx : lane);
    const double ay = fabs(__dsub_rn(yn, w.y));
    w.bok = nx >= 0 && dbits(ay) < dbits(s.d);
    w.b = __dsqrt_rn(__dsub_rn(s.d2, __dmul_rn(ay, ay)));
    if (!w.bok) w.nx = -1;
}

// Rare FP64 fix-ups, out of line: the compiler then never evaluates them on
// the common path (each FP64 instruction occupies the FP64 unit ~64 cycles).
__device__ __noinline__ double rp_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __noinline__ double rp_sub(double a, double b) { return __dsub_rn(a, b); }

// Each lane's step decided ahead, as the step would decide it, for the
// moment its disk becomes the active one (rp_prep): RP_PREP_OK when the
// predicted target is certain (the step's own test would find no candidate
// in doubt, the scan ends inside the window), with the target's lane and
// the scanned columns; the step then takes the lift whenever tau < D.
// Between slides the window changes only behind the active disk (a moved
// disk lands at contact with the next one), so what a lane's step reads --
// its disk, the disks after it, their owners and columns -- is as at the
// slide.
constexpr uint32_t RP_PREP_OK = 1u << 31;
constexpr uint32_t RP_PREP_CELL = 1u << 30;  // bits 16-20: the slot the moved disk takes

template <int C>
__device__ void rp_prep(const Dev &s, const StopK &sk, const RowChain &ch, const RowLane &w,
                        int nxr, int rnk, double &ptau, double &pxn, uint32_t &pinfo) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31, g = lane / C;
    const int v = (g - ch.gbase) & (G - 1);
    const bool occ = w.id != EMPTY;
    const int nx = w.nx;
    // the predicted target (the next disk in x order) and the disk after it
    const int src = nx >= 0 ? nx : lane;
    const double xn = __shfl_sync(FULL, w.x, src);
    const uint32_t ownn = __shfl_sync(FULL, w.own, src);
    const int tzn = __shfl_sync(FULL, (int)(dbits(w.t) != 0ull), src);
    const uint32_t skn = __shfl_sync(FULL, w.skp, src);
    const int nx2 = __shfl_sync(FULL, nxr, src);
    const int src2 = (nx >= 0 && nx2 >= 0) ? nx2 : lane;
    const double xn2 = __shfl_sync(FULL, w.x, src2);
    const int vn = ((src / C) - ch.gbase) & (G - 1);
    const int vn2 = ((src2 / C) - ch.gbase) & (G - 1);
    // window ranks (position, then x) of the disks of other chains
    const int R = v * C + rnk;
    const unsigned nsR = __reduce_or_sync(FULL, (occ && w.own != OWN_STATIC) ? (1u << R) : 0u);
    // lazy frame (a target with t != 0), and a target whose rows are in
    // reach (the row pass cancels there), are left to the step
    bool ok = occ && nx >= 0 && ownn == OWN_STATIC && !tzn && skn == RP_SKIP_ALL;
    // tau of the target, with the step's operations
    double dx = __dsub_rn(xn, w.x);
    const bool wl = ok && dneg(dx) && vn > v;
    if (__any_sync(FULL, wl) && wl) dx = rp_add(dx, s.L);
    double tau = __dsub_rn(dx, w.b);
    if (dneg(tau)) tau = 0.0;
    const unsigned long long cur = dbits(tau);
    // the stop rule with best = tau: the scan reaches the target's column and
    // stops inside the window
    const double fx = __dsub_rn(w.x, w.colx);
    const float fxf = d2f_trunc(fx);
    const float lim_f = __fadd_rn(d2f_trunc(tau), sk.epsf);
    const int mp = vn - v;
    int mstop = G;
    if (ok) {
        if (mp >= 1 && beyond_k(sk, mp, fx, fxf, lim_f, cur)) ok = false;
        for (int m = mp + 1; ok && m < G - v; ++m)
            if (beyond_k(sk, m, fx, fxf, lim_f, cur)) {
                mstop = m;
                break;
            }
        if (mstop >= G - v) ok = false;
    }
    // no other chain's disk after this one in the scanned columns (the
    // target included), and the next candidate's lower bound dx - d above tau
    // (every later one's is larger: RN is monotone)
    if (ok) {
        const int lim = (v + mstop) * C;
        const unsigned inrange = lim >= 32 ? ~0u : ((1u << lim) - 1u);
        const unsigned after = R >= 31 ? 0u : ~((2u << R) - 1u);
        if (nsR & inrange & after) ok = false;
    }
    const bool chk2 = ok && nx2 >= 0 && vn2 < v + mstop;
    if (__any_sync(FULL, chk2) && chk2) {
        double dx2 = __dsub_rn(xn2, w.x);
        if (dneg(dx2) && vn2 > v) dx2 = rp_add(dx2, s.L);
        const double sub2 = __dsub_rn(dx2, sk.d);
        if (dneg(sub2) || !(dbits(sub2) > cur)) ok = false;
    }
    // the moved disk's new cell: its own column (same slot) or the next one
    // (its lowest empty slot; that column is as at the slide)
    double xnew = __dadd_rn(w.x, tau);
    const bool wrap = ok && !(dbits(xnew) < dbits(s.L));
    if (__any_sync(FULL, wrap) && wrap) xnew = rp_sub(xnew, s.L);
    const unsigned long long xb = dbits(xnew);
    const int g1 = ((g + 1) & (G - 1)) * C;
    const unsigned long long xlo1 = shfl_u64(w.xlo, g1), xhi1 = shfl_u64(w.xhi, g1);
    const unsigned em = __ballot_sync(FULL, w.id == EMPTY);
    uint32_t cell = 0u;
    if (ok) {
        if (xb >= w.xlo && xb < w.xhi) {
            cell = RP_PREP_CELL | ((uint32_t)lane << 16);
        } else if (v + 1 < G && xb >= xlo1 && xb < xhi1) {
            const unsigned m1 = em & (((1u << C) - 1u) << g1);
            if (m1) cell = RP_PREP_CELL | ((uint32_t)(__ffs(m1) - 1) << 16);
        }
    }
    ptau = tau;
    pxn = xnew;
    pinfo = ok ? (RP_PREP_OK | cell | (uint32_t)nx | ((uint32_t)mstop << 8)) : 0u;
}

// The continuation's steps decided ahead where D does not enter: the
// target (static, rows out of reach, t_i + tau moves the disk within its
// slot) and tau, the disk's fx, its window rank, and whether the candidate
// after the target has its lower bound above tau. The scan to D, the owners
// and the cells' holders over it, and Eq. 2 are the batch's, per step.
constexpr uint32_t RC_PREP_OK = 1u << 31;
constexpr uint32_t RC_PREP_NX2OK = 1u << 30;

template <int C>
__device__ void rc_prep(const Dev &s, const RowChain &ch, const RowLane &w, int nxr, int rnk,
                        double &ptau, double &pxn, double &pfx, int &pR, unsigned &nsR,
                        uint32_t &pinfo, float *thrf, float &pxf, float &ptf) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31, g = lane / C;
    const int v = (g - ch.gbase) & (G - 1);
    const bool occ = w.id != EMPTY;
    const int nx = w.nx;
    const int src = nx >= 0 ? nx : lane;
    const double xn = __shfl_sync(FULL, w.x, src);
    const uint32_t ownn = __shfl_sync(FULL, w.own, src);
    const uint32_t skn = __shfl_sync(FULL, w.skp, src);
    const int nx2 = __shfl_sync(FULL, nxr, src);
    const int src2 = (nx >= 0 && nx2 >= 0) ? nx2 : lane;
    const double xn2 = __shfl_sync(FULL, w.x, src2);
    const int vn = ((src / C) - ch.gbase) & (G - 1);
    const int vn2 = ((src2 / C) - ch.gbase) & (G - 1);
    pR = v * C + rnk;
    nsR = __reduce_or_sync(FULL, (occ && w.own != OWN_STATIC) ? (1u << pR) : 0u);
    bool ok = occ && nx >= 0 && ownn == OWN_STATIC && skn == RP_SKIP_ALL;
    double dx = __dsub_rn(xn, w.x);
    const bool wl = ok && dneg(dx) && vn > v;
    if (__any_sync(FULL, wl) && wl) dx = rp_add(dx, s.L);
    double tau = __dsub_rn(dx, w.b);
    // (a negative dx - b is the step's: Eq. 2 there reads the unclamped value)
    if (dneg(tau)) {
        tau = 0.0;
        ok = false;
    }
    pfx = __dsub_rn(w.x, w.colx);
    // FP32 images: the stop rule's thr(m) = ((m a) - fx) - d for m = 1, 2, 3
    // (as beyond_k forms it), x and t (truncated)
    {
        const float fxf = d2f_trunc(pfx);
#pragma unroll
        for (int m = 1; m <= 3; ++m)
            thrf[m - 1] = __fsub_rn(__fsub_rn(__fmul_rn(__int2float_rn(m), s.af), fxf), s.df);
        pxf = d2f_trunc(w.x);
        ptf = d2f_trunc(w.t);
    }
    bool nx2ok = true;
    const bool chk2 = ok && nx2 >= 0;
    if (__any_sync(FULL, chk2) && chk2) {
        double dx2 = __dsub_rn(xn2, w.x);
        if (dneg(dx2) && vn2 > v) dx2 = rp_add(dx2, s.L);
        const double sub2 = __dsub_rn(dx2, s.d);
        nx2ok = !dneg(sub2) && dbits(sub2) > dbits(tau);
    }
    // the moved disk stays in its slot (else the step below)
    double xnew = __dadd_rn(w.x, tau);
    const bool wrap = ok && !(dbits(xnew) < dbits(s.L));
    if (__any_sync(FULL, wrap) && wrap) xnew = rp_sub(xnew, s.L);
    if (ok && !(dbits(xnew) >= w.xlo && dbits(xnew) < w.xhi)) ok = false;
    ptau = tau;
    pxn = xnew;
    const uint32_t p2 = (nx2 >= 0 && ok) ? (uint32_t)vn2 : 31u;
    pinfo = ok ? (RC_PREP_OK | (nx2ok ? RC_PREP_NX2OK : 0u) | (uint32_t)nx | (p2 << 8)) : 0u;
}

struct RowStep {
    int lift;          // 1: lift onto lane p; 0: stall
    int p;             // lane of the target
    double tau;        // tau* or D
    int mstop;         // scanned columns: 0 .. mstop - 1 from the active disk's
    int nonstatic;     // Remark 10 (as in scan_step)
    uint32_t ns_owner;
    int overflow;      // the scan does not end inside the window
    int viol;          // CONT: a scanned corridor disk fails Eq. 2
};

// The step evaluated exactly over the window, lane by lane, with the
// operations of scan_step (PASS1 mode, or CONT: the scan runs to D and Eq. 2
// is checked on every scanned corridor disk) and its stop rule column by
// column. vi: window position of the active disk's column.
template <int C, bool CONT = false>
__device__ RowStep rp_exact(const Dev &s, const StopK &sk, const RowChain &ch, const RowLane &w,
                            int vi, float fxf) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31, g = lane / C;
    const int v = (g - ch.gbase) & (G - 1);
    const bool cand = w.id != EMPTY && w.id != ch.i && v >= vi;
    const bool st = w.own == OWN_STATIC;
    const double ay = fabs(__dsub_rn(w.y, ch.yi));
    const bool inc = dbits(ay) < dbits(s.d);
    const bool corr = cand && st && inc;
    const bool ncs = cand && !st && inc;
    const double b = __dsqrt_rn(__dsub_rn(s.d2, __dmul_rn(ay, ay)));
    double dx = __dsub_rn(w.x, ch.xi);
    const bool neg = dneg(dx);
    // a disk behind the active disk in its own column is more than L - 2a
    // ahead and beyond reach (D < L - 3a here); elsewhere a negative dx means
    // the window crossed the box edge: the forward image adds L (for another
    // chain's disk in any column, as scan_step does)
    const bool drop = neg && v == vi;
    const bool wl = (corr && neg && !drop) || (ncs && neg);
    if (__any_sync(FULL, wl) && wl) dx = __dadd_rn(dx, s.L);
    double tau = INFINITY;
    if (corr && !drop) {
        tau = __dsub_rn(dx, b);
        if (dneg(tau)) tau = 0.0;
    }
    // lazy frame: a disk that became static after the active disk passed it
    // is one lap away
    const bool tnz = tau != INFINITY && dbits(w.t) != 0ull;
    bool hzv = false;
    if (__any_sync(FULL, tnz)) {
        const double sum = __dadd_rn(ch.ti, tau);
        const bool behind = tnz && dbits(sum) < dbits(w.t);
        // the horizon condition t_i + tau > t_j (Eq. 2, strict)
        if (CONT) hzv = tnz && !(dbits(sum) > dbits(w.t));
        if (__any_sync(FULL, behind) && behind) tau = __dadd_rn(tau, s.L);
    }
    // another chain's active or stalled disk: time of flight and Eq. 2
    unsigned long long nt = INF_BITS;
    uint32_t no = NONE;
    bool hv = false;
    if (__any_sync(FULL, ncs)) {
        if (ncs) {
            double tn = __dsub_rn(dx, b);
            if (dneg(tn)) tn = 0.0;
            nt = dbits(tn);
            no = w.own & OWN_CHAIN;
            if (dbits(w.t) != 0ull && !(dbits(__dadd_rn(ch.ti, tn)) > dbits(w.t))) hv = true;
        }
    }
    // (tau, j) and (tn, owner) minima of each column (an aligned group of C lanes)
    unsigned long long ct = dbits(tau);
    uint32_t cj = ct != INF_BITS ? w.id : NONE;
    int cl = lane;
#pragma unroll
    for (int o = 1; o < C; o <<= 1) {
        const unsigned long long t2 = shfl_xor_u64(ct, o);
        const uint32_t j2 = __shfl_xor_sync(FULL, cj, o);
        const int l2 = __shfl_xor_sync(FULL, cl, o);
        if (t2 < ct || (t2 == ct && j2 < cj)) {
            ct = t2;
            cj = j2;
            cl = l2;
        }
        const unsigned long long n2 = shfl_xor_u64(nt, o);
        const uint32_t o2 = __shfl_xor_sync(FULL, no, o);
        if (n2 < nt || (n2 == nt && o2 < no)) {
            nt = n2;
            no = o2;
        }
    }
    const unsigned hvm = __ballot_sync(FULL, hv);
    const unsigned vm = __ballot_sync(FULL, hzv);
    // columns in order, with the scan's stop rule
    unsigned long long cur = dbits(ch.D);
    float lim_f = __fadd_rn(d2f_trunc(ch.D), s.epsf);
    unsigned long long best = INF_BITS, ns_t = INF_BITS;
    uint32_t bj = NONE, ns_o = NONE;
    int bl = -1;
    bool hvany = false, vany = false;
    int m = 0;
    for (; vi + m < G; ++m) {
        if (m >= 1 && beyond_k(sk, m, ch.fx, fxf, lim_f, cur)) break;
        const int src = ((ch.gbase + vi + m) & (G - 1)) * C;
        const unsigned long long t2 = shfl_u64(ct, src);
        const uint32_t j2 = __shfl_sync(FULL, cj, src);
        const int l2 = __shfl_sync(FULL, cl, src);
        if (t2 < best || (t2 == best && j2 < bj)) {
            best = t2;
            bj = j2;
            bl = l2;
        }
        if (!CONT && t2 < cur) {
            cur = t2;
            lim_f = __fadd_rn(d2f_trunc(__longlong_as_double((long long)cur)), s.epsf);
        }
        const unsigned long long n2 = shfl_u64(nt, src);
        const uint32_t o2 = __shfl_sync(FULL, no, src);
        if (n2 < ns_t || (n2 == ns_t && o2 < ns_o)) {
            ns_t = n2;
            ns_o = o2;
        }
        hvany |= ((hvm >> src) & ((1u << C) - 1u)) != 0u;
        vany |= ((vm >> src) & ((1u << C) - 1u)) != 0u;
    }
    RowStep r;
    r.viol = vany;
    r.overflow = vi + m >= G;
    r.mstop = m;
    r.nonstatic = hvany || ns_t < dbits(ch.D);
    r.ns_owner = ns_o;
    if (best < dbits(ch.D)) {
        r.lift = 1;
        r.p = bl;
        r.tau = __longlong_as_double((long long)best);
    } else {
        r.lift = 0;
        r.p = -1;
        r.tau = ch.D;
    }
    return r;
}

__device__ __forceinline__ void red_min_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v));
}
__device__ __forceinline__ void red_min_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v));
}
__device__ __forceinline__ void red_max_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v));
}

// Fire-and-forget claims of the columns the step scans beyond those already
// claimed: the active row strongly, the two rows out of reach weakly. Lane
// 4e + r covers row r - 1 (r < 3) of the columns front + 1 + e, e + 8, ...;
// rowb is that row's first cell (each lane's own, fixed for the chain).
__device__ __forceinline__ void rp_claim(const Dev &s, RowChain &ch, int first, int last,
                                         uint32_t rowb) {
    if (last <= ch.front) return;
    const int lane = threadIdx.x & 31, dr = lane & 3;
    if (dr < 3) {
        const uint32_t cm = (uint32_t)ch.c + 1u;
        for (int o = ch.front + 1 + (lane >> 2); o <= last; o += 8) {
            const unsigned long long key = rp_key(ch.c, ch.ti, o - first, dr != 1);
            int col = ch.u0 + o;
            if (col >= s.nc) col -= s.nc;
            const uint32_t cell = rowb + (uint32_t)col;
            red_min_u64(s.ckey + cell, key);
            red_min_u32(s.camin + cell, cm);
            red_max_u32(s.camax + cell, cm);
        }
    }
    ch.front = last;
}


// The stop rule for the column offsets 1 .. mmax - 1 from the active disk's
// column, one per lane: bit m is beyond(m, cur) (FP32 image; exact FP64 for
// the lanes it leaves undecided).
__device__ __forceinline__ unsigned rp_stop_mask(const StopK &sk, double fx, float fxf,
                                                 unsigned long long cur, int mmax) {
    const int lane = threadIdx.x & 31;
    const float lim_f = __fadd_rn(d2f_trunc(__longlong_as_double((long long)cur)), sk.epsf);
    bool bey = false, und = false;
    if (lane >= 1 && lane < mmax) {
        if (!(sk.stop_e > 0.f)) {
            und = true;
        } else {
            const float thr_f =
                __fsub_rn(__fsub_rn(__fmul_rn((float)lane, sk.af), fxf), sk.df);
            const float diff = __fsub_rn(thr_f, lim_f);
            if (diff > sk.stop_e)
                bey = true;
            else if (!(diff < -sk.stop_e))
                und = true;
        }
    }
    if (__any_sync(FULL, und) && und) bey = beyond_exact(sk.a, sk.d, sk.eps, lane, fx, cur);
    return __ballot_sync(FULL, bey);
}

// The speculative pass of chain c over the window [tw, tend) (see the head of
// this file). Returns false if it had to cancel the system's row pass.
template <int C>
__device__ bool row_pass_chain(const Dev &s, int c, double tw, double tend) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31, gme = lane / C;
    if (s.status[c] != ST_RUNNING) {
        if (lane == 0) s.rp_front[c] = -1;  // claims nothing
        return true;
    }
    const StopK sk = stopk_of(s);
    const double dd = s.d, LL = s.L;
    const int cap = s.cap;
    // the window must never reload a column the chain already passed (its
    // cells changed in the warp only): its last column stays below offset nc
    const int far_cols = s.nc;
    RowChain ch;
    ch.c = c;
    const uint32_t aloc = s.aloc[c];
    if (lane == 0) s.rp_start[c] = aloc;
    const uint32_t cell0 = aloc / C;
    ch.row = (int)(cell0 / (uint32_t)s.nc);
    ch.u0 = (int)(cell0 % (uint32_t)s.nc);
    ch.wbase = 0;
    ch.gbase = 0;
    ch.i = s.ci[c];
    ch.ti = s.tc[c];
    ch.D = s.D[c];
    ch.front = -1;
    ch.nrec0 = s.nrec[c];
    ch.n = 0;
    ch.lifts = 0;
    uint32_t rowb;
    {
        int r = ch.row + (lane & 3) - 1;
        if (r < 0) r += s.nc;
        if (r >= s.nc) r -= s.nc;
        rowb = (uint32_t)r * (uint32_t)s.nc;
    }
    RowLane w;
    rp_load<C>(s, ch, w, gme);
    rp_prefetch<C>(s, ch, G);
    ch.li = (int)(aloc % C);  // position 0 is group 0
    int vi = 0;
    // claims of prepared steps, held until their column leaves the window:
    // lane q < 3 of a column's group claims row q - 1 of it (the key of the
    // first step that scanned it, as rp_claim computes it)
    const int qrow = lane % C;
    uint32_t prowb;
    {
        int r = ch.row + qrow - 1;
        if (r < 0) r += s.nc;
        if (r >= s.nc) r -= s.nc;
        prowb = (uint32_t)r * (uint32_t)s.nc;
    }
    unsigned long long pk = ~0ull;
    auto flush = [&](int vmax) {  // the held claims of window positions < vmax
        const int vq = (gme - ch.gbase) & (G - 1);
        if (pk != ~0ull && vq < vmax) {
            int col = ch.u0 + ch.wbase + vq;
            while (col >= s.nc) col -= s.nc;
            const uint32_t cell = prowb + (uint32_t)col;
            const uint32_t cm = (uint32_t)c + 1u;
            red_min_u64(s.ckey + cell, pk);
            red_min_u32(s.camin + cell, cm);
            red_max_u32(s.camax + cell, cm);
            pk = ~0ull;
        }
    };
    ch.xi = __shfl_sync(FULL, w.x, ch.li);
    ch.yi = __shfl_sync(FULL, w.y, ch.li);
    ch.iskp = __shfl_sync(FULL, w.skp, ch.li);
    ch.fx = __dsub_rn(ch.xi, __shfl_sync(FULL, w.colx, ch.li));
    double ptau, pxn;  // this lane's step, decided ahead (rp_prep)
    uint32_t pinfo;
    {
        int nxr, rnk;
        rp_links<C>(s, ch, w, &nxr, &rnk);
        rp_prep<C>(s, sk, ch, w, nxr, rnk, ptau, pxn, pinfo);
    }
    int nx = __shfl_sync(FULL, w.nx, ch.li);
    double bnx = __shfl_sync(FULL, w.b, ch.li);
    // slides the window by h columns (the active disk's column moves to
    // position vi - h); false if the window would reach the start column
    auto slide = [&](int h) -> bool {
        if (ch.wbase + h + G > far_cols) return false;
        flush(h);
        const int v0 = (gme - ch.gbase) & (G - 1);
        ch.wbase += h;
        ch.gbase = (ch.gbase + h) & (G - 1);
        if (v0 < h) rp_load<C>(s, ch, w, v0 + G - h);
        rp_prefetch<C>(s, ch, ch.wbase + G);
        vi -= h;
        int nxr, rnk;
        rp_links<C>(s, ch, w, &nxr, &rnk);
        rp_prep<C>(s, sk, ch, w, nxr, rnk, ptau, pxn, pinfo);
        nx = __shfl_sync(FULL, w.nx, ch.li);
        bnx = __shfl_sync(FULL, w.b, ch.li);
        return true;
    };
    int end = RP_END_PAUSE;
    uint32_t ns_owner = NONE;
    bool ok = ch.iskp == RP_SKIP_ALL;
    // slide once the active column reaches SLIDE_AT: a step's scan reads its
    // own column and the next one or two (a scan that would leave the window
    // slides first, below)
    constexpr int SLIDE_AT = G > 4 ? G - 2 : G / 2;
    auto v_of_lane = [&](int l) { return ((l / C) - ch.gbase) & (G - 1); };
    while (ok) {
        if (vi >= SLIDE_AT && !slide(vi)) {
            ok = false;
            break;
        }
        const int v = (gme - ch.gbase) & (G - 1);
        // a batch of prepared steps that keep the moved disk in its slot: the
        // chain through them in uniform registers (the target, tau, the
        // claims, t_i + tau and D - tau), then each step's record and window
        // update by the lane of the disk that moved, all at once
        {
            int lk = ch.li, K = 0, front = ch.front;
            double t = ch.ti, D = ch.D;
            bool pause = false;
            int my_k = -1, my_front = 0;
            double my_t = 0.0, my_tn = 0.0, my_dn = 0.0;
            for (;;) {
                const uint32_t info = __shfl_sync(FULL, pinfo, lk);
                if ((info & (RP_PREP_OK | RP_PREP_CELL)) != (RP_PREP_OK | RP_PREP_CELL) ||
                    (int)((info >> 16) & 31u) != lk)
                    break;
                const int vk = ((lk / C) - ch.gbase) & (G - 1);
                if (K > 0 && vk >= SLIDE_AT) break;
                if (ch.nrec0 + ch.n + K >= cap) break;
                const double tau = __shfl_sync(FULL, ptau, lk);
                if (!(dbits(tau) < dbits(D))) break;  // a stall: the step below
                const double tn = __dadd_rn(t, tau);
                if (dbits(tn) < dbits(tw)) break;     // (never: the step below reports it)
                const int last = ch.wbase + vk + (int)((info >> 8) & 31u) - 1;
                if (last > front) {
                    const int oabs = ch.wbase + v;
                    if (qrow < 3 && oabs > front && oabs <= last)
                        pk = rp_key(c, t, v - vk, qrow != 1);
                    front = last;
                }
                if (!(dbits(tn) < dbits(tend))) {  // pauses at the window end
                    pause = true;
                    break;
                }
                const double dn = __dsub_rn(D, tau);
                if (lane == lk) {
                    my_k = K;
                    my_t = t;
                    my_tn = tn;
                    my_dn = dn;
                    my_front = front;
                }
                t = tn;
                D = dn;
                ++K;
                lk = (int)(info & 31u);
            }
            if (K > 0) {
                // the records, with the targets' fields as they were
                const int nxl = w.nx;
                const int srcp = my_k >= 0 ? nxl : lane;
                const double xp = __shfl_sync(FULL, w.x, srcp);
                const double tp = __shfl_sync(FULL, w.t, srcp);
                const uint32_t idp = __shfl_sync(FULL, w.id, srcp);
                if (my_k >= 0) {
                    const uint32_t from = rp_loc_of<C>(s, ch, lane);
                    const uint32_t jloc = rp_loc_of<C>(s, ch, nxl);
                    const uint32_t e = (uint32_t)(ch.nrec0 + ch.n + my_k);
                    ulonglong2 *q = (ulonglong2 *)rec_at(s, c, (int32_t)e);
                    q[0] = make_ulonglong2((unsigned long long)w.id | ((unsigned long long)from << 32),
                                           (unsigned long long)from | ((unsigned long long)idp << 32));
                    q[1] = make_ulonglong2((unsigned long long)jloc | ((unsigned long long)e << 32),
                                           (unsigned long long)(uint32_t)my_front << 32);
                    q[2] = make_ulonglong2(dbits(w.x), dbits(my_t));
                    q[3] = make_ulonglong2(dbits(tp), dbits(my_tn));
                    q[4] = make_ulonglong2(dbits(ptau), dbits(pxn));
                    q[5] = make_ulonglong2(dbits(xp), dbits(my_dn));
                    // the disk moved within its slot and is static now
                    w.x = pxn;
                    w.t = my_tn;
                    w.own = OWN_STATIC;
                    w.nx = -1;
                    w.bok = 0;
                } else if (lane == lk) {
                    w.t = t;
                    w.own = OWN_ACTIVE | (uint32_t)c;
                }
                ch.n += K;
                ch.lifts += K;
                ch.front = front;
                ch.li = lk;
                ch.i = __shfl_sync(FULL, w.id, lk);
                ch.xi = __shfl_sync(FULL, w.x, lk);
                ch.yi = __shfl_sync(FULL, w.y, lk);
                ch.ti = t;
                ch.D = D;
                ch.fx = __dsub_rn(ch.xi, __shfl_sync(FULL, w.colx, lk));
                vi = v_of_lane(lk);
                nx = __shfl_sync(FULL, w.nx, lk);
                bnx = __shfl_sync(FULL, w.b, lk);
            } else if (pause) {
                ch.front = front;
            }
            if (pause) break;
            if (K > 0) continue;
        }
        RowStep rs;
        // the step decided at the slide (the common case), else below
        bool fast = false;
        const uint32_t pinf = __shfl_sync(FULL, pinfo, ch.li);
        {
            if (pinf & RP_PREP_OK) {
                const double tp = __shfl_sync(FULL, ptau, ch.li);
                if (dbits(tp) < dbits(ch.D)) {
                    fast = true;
                    rs.lift = 1;
                    rs.p = (int)(pinf & 31u);
                    rs.tau = tp;
                    rs.mstop = (int)((pinf >> 8) & 31u);
                    rs.nonstatic = 0;
                    rs.ns_owner = NONE;
                    rs.overflow = 0;
                    rs.viol = 0;
                }
            }
        }
        if (!fast) {
        const float fxf = d2f_trunc(ch.fx);
        const bool occ = w.id != EMPTY;
        // prediction: the next disk in x order (nx), b towards it cached
        const int pp = nx;
        double dx = __dsub_rn(w.x, ch.xi);
        const bool neg = dneg(dx);
        const bool wl = occ && neg && v > vi;
        if (__any_sync(FULL, wl) && wl) dx = rp_add(dx, LL);
        // tau of the predicted target, dx - d (a lower bound of tau) elsewhere
        const double sub = __dsub_rn(dx, lane == pp ? bnx : dd);
        double taup = INFINITY;
        if (pp >= 0) {
            taup = __shfl_sync(FULL, sub, pp);
            if (dneg(taup)) taup = 0.0;
        }
        const bool lift = pp >= 0 && dbits(taup) < dbits(ch.D);
        const unsigned long long cur = lift ? dbits(taup) : dbits(ch.D);
        const unsigned smask = rp_stop_mask(sk, ch.fx, fxf, cur, G - vi);
        const int mp = lift ? (((pp / C) - ch.gbase) & (G - 1)) - vi : 0;
        const int mmin = lift ? mp + 1 : 1;
        const unsigned above = mmin < 32 ? smask & ~((1u << mmin) - 1u) : 0u;
        int mstop = above ? __ffs(above) - 1 : G - vi;
        bool exact = mstop >= G - vi || (lift && (mp < 0 || (mp >= 1 && ((smask >> mp) & 1u))));
        {
            const bool scanned = occ && v >= vi && v < vi + mstop;
            const bool cnd = scanned && w.id != ch.i && !(neg && v == vi) && !(lift && lane == pp);
            bool bad = cnd && (w.own != OWN_STATIC || dneg(sub) ||
                               (lift ? !(dbits(sub) > cur) : !(dbits(sub) >= cur)));
            // the target must be static (another chain's active or stalled
            // disk stops the chain, Remark 10) and ahead in the lazy frame
            if (lift && lane == pp) {
                if (w.own != OWN_STATIC)
                    bad = true;
                else if (dbits(w.t) != 0ull && dbits(rp_add(ch.ti, taup)) < dbits(w.t))
                    bad = true;
            }
            if (__any_sync(FULL, bad)) exact = true;
        }
        if (exact) {
            rs = rp_exact<C>(s, sk, ch, w, vi, fxf);
            if (rs.overflow) {
                if (vi > 0 && slide(vi)) continue;
                ok = false;
                break;
            }
        } else {
            rs.lift = lift;
            rs.p = lift ? pp : -1;
            rs.tau = lift ? taup : ch.D;
            rs.mstop = mstop;
            rs.nonstatic = 0;
            rs.ns_owner = NONE;
            rs.overflow = 0;
            rs.viol = 0;
        }
        }
        if (fast) {
            const int last = ch.wbase + vi + rs.mstop - 1;
            if (last > ch.front) {
                const int oabs = ch.wbase + v;
                if (qrow < 3 && oabs > ch.front && oabs <= last)
                    pk = rp_key(c, ch.ti, v - vi, qrow != 1);
                ch.front = last;
            }
        } else {
            rp_claim(s, ch, ch.wbase + vi, ch.wbase + vi + rs.mstop - 1, rowb);
        }
        if (rs.nonstatic) {
            end = RP_END_NONSTATIC;
            ns_owner = rs.ns_owner;
            break;
        }
        // t_i + tau, x_i + tau, D - tau and the target's offset in its cell:
        // one lane-parallel addition
        const int p = rs.p;
        const int pe = p >= 0 ? p : 0;
        const int a0 = (pe + 1) & 31, a1 = (pe + 2) & 31, a2 = (pe + 3) & 31;
        double opa = ch.D, opb = -rs.tau;
        if (lane == a0) {
            opa = ch.ti;
            opb = rs.tau;
        } else if (lane == a1) {
            opa = ch.xi;
            opb = rs.tau;
        } else if (p >= 0 && lane == p) {
            opa = w.x;
            opb = -w.colx;
        }
        const double sum = __dadd_rn(opa, opb);
        const double tnew = __shfl_sync(FULL, sum, a0);
        double xnew = __shfl_sync(FULL, sum, a1);
        if (!(dbits(tnew) < dbits(tend))) break;  // pauses at the window end
        if (dbits(tnew) < dbits(tw) && lane == 0) {
            atomicAdd(s.lc + LC_ORDER, 1ull);
            diag(s, 10, tw, c, ch.i, rs.p, ch.ti, rs.tau);
        }
        if (ch.nrec0 + ch.n >= cap) {
            ok = false;
            break;
        }
        if (dbits(xnew) >= dbits(LL)) xnew = rp_sub(xnew, LL);
        // the moved disk's new cell: a column of the window at or after its own
        // (decided at the slide for a prepared step)
        int ln = ch.li;
        if (fast && (pinf & RP_PREP_CELL)) {
            ln = (int)((pinf >> 16) & 31u);
        } else {
            const unsigned long long xb = dbits(xnew);
            const unsigned hm =
                __ballot_sync(FULL, lane % C == 0 && v >= vi && xb >= w.xlo && xb < w.xhi);
            if (!hm) {
                ok = false;
                break;
            }
            const int gn = (__ffs(hm) - 1) / C;
            if (gn != ch.li / C) {
                const unsigned em =
                    __ballot_sync(FULL, w.id == EMPTY) & (((1u << C) - 1u) << (gn * C));
                if (!em) {
                    ok = false;
                    break;
                }
                ln = __ffs(em) - 1;
            }
        }
        // the event record (as commit_step writes it; pad: the scan's last
        // column): the target's lane stores the words that carry its fields,
        // lane 0 the others (all of them for a stall)
        const uint32_t from = rp_loc_of<C>(s, ch, ch.li);
        const uint32_t to = rp_loc_of<C>(s, ch, ln);
        const uint32_t jloc = rs.lift ? rp_loc_of<C>(s, ch, p) : 0u;
        {
            const double dnew = __shfl_sync(FULL, sum, a2);
            ulonglong2 *q = (ulonglong2 *)rec_at(s, c, ch.nrec0 + ch.n);
            const bool tl = rs.lift ? lane == p : lane == 0;
            if (tl) {
                const uint32_t jid = rs.lift ? w.id : NONE;
                q[0] = make_ulonglong2((unsigned long long)ch.i | ((unsigned long long)from << 32),
                                       (unsigned long long)to | ((unsigned long long)jid << 32));
                q[3] = make_ulonglong2(rs.lift ? dbits(w.t) : 0ull, dbits(tnew));
                q[5] = make_ulonglong2(rs.lift ? dbits(w.x) : 0ull, rs.lift ? dbits(dnew) : 0ull);
            }
            if (lane == 0) {
                q[1] = make_ulonglong2(
                    (unsigned long long)jloc |
                        ((unsigned long long)(uint32_t)(ch.nrec0 + ch.n) << 32),
                    (unsigned long long)(uint32_t)ch.front << 32);
                q[2] = make_ulonglong2(dbits(ch.xi), dbits(ch.ti));
                q[4] = make_ulonglong2(dbits(rs.tau), dbits(xnew));
            }
            ch.D = rs.lift ? dnew : 0.0;
        }
        ++ch.n;
        // the window follows the event
        double xj = 0.0, yj = 0.0, fxn = 0.0;
        uint32_t jid = NONE;
        if (rs.lift) {
            xj = __shfl_sync(FULL, w.x, p);
            yj = __shfl_sync(FULL, w.y, p);
            jid = __shfl_sync(FULL, w.id, p);
            fxn = __shfl_sync(FULL, sum, p);
            if (lane == p) {
                w.t = tnew;
                w.own = OWN_ACTIVE | (uint32_t)c;
            }
        }
        if (ln != ch.li && lane == ch.li) w.id = EMPTY;
        if (lane == ln) {
            w.id = ch.i;
            w.x = xnew;
            w.y = ch.yi;
            w.t = tnew;
            w.own = rs.lift ? OWN_STATIC : (OWN_STALLED | (uint32_t)c);
            w.skp = ch.iskp;
            w.nx = -1;
            w.bok = 0;
        }
        if (!rs.lift) {
            end = RP_END_STALL;
            ch.li = ln;
            ch.xi = xnew;
            ch.ti = tnew;
            break;
        }
        ++ch.lifts;
        // the target's rows must be out of reach too (else cancel)
        if (__ballot_sync(FULL, lane == p && w.skp != RP_SKIP_ALL)) {
            ok = false;
            break;
        }
        nx = __shfl_sync(FULL, w.nx, p);
        bnx = __shfl_sync(FULL, w.b, p);
        ch.i = jid;
        ch.li = p;
        vi = (((p / C) - ch.gbase) & (G - 1));
        ch.xi = xj;
        ch.yi = yj;
        ch.ti = tnew;
        ch.fx = fxn;
    }
    if (!ok) return false;
    flush(G);
    // the end of the speculative run, for row_resolve_chain
    if (lane == 0) {
        s.rp_n[c] = ch.n;
        s.rp_front[c] = ch.front;
        s.rp_end[c] = end;
        s.rp_partner[c] = (end == RP_END_NONSTATIC && ns_owner < (uint32_t)s.k) ? (int32_t)ns_owner : -1;
        s.rp_ci[c] = ch.i;
        s.rp_tc[c] = ch.ti;
        s.rp_D[c] = ch.D;
        s.rp_aloc[c] = rp_loc_of<C>(s, ch, ch.li);
    }
    return true;
}

// The claim arrays back to empty over the cells chain c claimed in the row
// pass (rows row - 1 .. row + 1, columns 0 .. rp_front from its start).
template <int C>
__device__ void row_reset_chain(const Dev &s, int c) {
    const int front = s.rp_front[c];
    if (front < 0) return;
    const int lane = threadIdx.x & 31, nc = s.nc;
    const uint32_t cell0 = s.rp_start[c] / C;
    const int row = (int)(cell0 / (uint32_t)nc), u0 = (int)(cell0 % (uint32_t)nc);
    unsigned long long *const ck = s.ckey;
    uint32_t *const mn = s.camin, *const mx = s.camax;
    for (int e = lane; e < 3 * (front + 1); e += 32) {
        const int o = e / 3;
        int col = u0 + o;
        if (col >= nc) col -= nc;
        int r = row + e % 3 - 1;
        if (r < 0) r += nc;
        if (r >= nc) r -= nc;
        const uint32_t cell = (uint32_t)r * (uint32_t)nc + (uint32_t)col;
        ck[cell] = ~0ull;
        mn[cell] = ~0u;
        mx[cell] = 0u;
    }
}

// After the pass: the first cell another chain holds, the events published
// before it, the chain's state, the claim words and the flag.
template <int C>
__device__ void row_resolve_chain(const Dev &s, int c, double tw) {
    const int lane = threadIdx.x & 31, nc = s.nc;
    if (c == 0 && lane == 0) atomicAdd(s.lc + LC_ROWWIN, 1ull);
    if (s.status[c] != ST_RUNNING) return;
    const uint32_t aloc = s.aloc[c];
    const uint32_t cell0 = aloc / C;
    const int row = (int)(cell0 / (uint32_t)nc), u0 = (int)(cell0 % (uint32_t)nc);
    const int n = s.rp_n[c], front = s.rp_front[c], end = s.rp_end[c];
    const int32_t nrec0 = s.nrec[c];
    // columns 0 .. front: holder of the active row's cell, two claimants anywhere
    int lost = -1;
    uint32_t holder = NONE;
    bool over = false;
    for (int base = 0; base <= front; base += 32) {
        const int o = base + lane;
        const bool valid = o <= front;
        bool mine = true;
        uint32_t hchain = NONE;
        bool ov = false;
        if (valid) {
            int col = u0 + o;
            if (col >= nc) col -= nc;
#pragma unroll
            for (int dr = 0; dr < 3; ++dr) {
                int r = row + dr - 1;
                if (r < 0) r += nc;
                if (r >= nc) r -= nc;
                const uint32_t cell = (uint32_t)r * (uint32_t)nc + (uint32_t)col;
                const unsigned long long key = __ldcg(s.ckey + cell);
                const uint32_t hc = (uint32_t)(key & RP_KEY_CHAIN);
                if (__ldcg(s.camin + cell) != __ldcg(s.camax + cell)) ov = true;
                s.claim[cell] = (hc + 1u) | ((key & RP_WEAK) ? CLAIM_WEAK : 0u);
                if (dr == 1) {
                    mine = hc == (uint32_t)c;
                    hchain = hc;
                }
            }
        }
        over |= __any_sync(FULL, ov);
        const unsigned lm = __ballot_sync(FULL, valid && !mine);
        if (lost < 0 && lm) {
            const int src = __ffs(lm) - 1;
            lost = base + src;
            holder = __shfl_sync(FULL, hchain, src);
        }
    }
    // the first record whose scan reached the lost column (n if only the
    // final scan did)
    int sfail = n;
    if (lost >= 0) {
        for (int e0 = 0; e0 < n; e0 += 32) {
            const int e = e0 + lane;
            const bool hit = e < n && (int)rec_at(s, c, nrec0 + e)->pad >= lost;
            const unsigned hm = __ballot_sync(FULL, hit);
            if (hm) {
                sfail = e0 + __ffs(hm) - 1;
                break;
            }
        }
    }
    // publish records 0 .. sfail - 1: their final effect, one record per
    // lane. Each record's disk moved once (the chain only moves forward), its
    // destination was an empty slot, and a target's own record (the next one)
    // rewrites it: so the slots vacated by a cell change are emptied first,
    // then every record writes its disk's new slot, and the target of the
    // last one becomes the chain's active disk. (A vacated slot keeps its
    // other fields: an empty slot's fields are never read.)
    int pub_lifts = 0;
    for (int e0 = 0; e0 < sfail; e0 += 32) {
        const int e = e0 + lane;
        if (e < sfail) {
            const Rec &q = *rec_at(s, c, nrec0 + e);
            if (q.to != q.from) s.cid[q.from] = EMPTY;
        }
    }
    __syncwarp();
    for (int e0 = 0; e0 < sfail; e0 += 32) {
        const int e = e0 + lane;
        uint32_t rj = NONE;
        if (e < sfail) {
            const Rec &q = *rec_at(s, c, nrec0 + e);
            const uint32_t i = q.i, from = q.from, to = q.to, jl = q.jloc;
            const double x = q.xi, t = q.t;
            rj = q.j;
            const uint32_t own = rj != NONE ? OWN_STATIC : (OWN_STALLED | (uint32_t)c);
            if (to != from) {
                const double y = s.cy[from];
                const uint8_t skp = s.cskp[from];
                s.cx[to] = x;
                s.cy[to] = y;
                s.cskp[to] = skp;
                s.ct[to] = t;
                s.cown[to] = own;
                s.cid[to] = i;
            } else {
                s.cx[from] = x;
                s.ct[from] = t;
                s.cown[from] = own;
            }
            if (e == sfail - 1 && rj != NONE) {
                s.cown[jl] = OWN_ACTIVE | (uint32_t)c;
                s.ct[jl] = t;
            }
        }
        pub_lifts += __popc(__ballot_sync(FULL, e < sfail && rj != NONE));
    }
    __syncwarp();
    // the chain's state
    const bool blocked = lost >= 0 || end == RP_END_NONSTATIC;
    if (lane == 0) {
        int st;
        uint32_t al, id;
        double tc, D;
        int32_t partner = -1;
        if (sfail < n) {
            const Rec &q = *rec_at(s, c, nrec0 + sfail);
            al = q.from;
            id = q.i;
            tc = q.ti_old;
            D = sfail > 0 ? rec_at(s, c, nrec0 + sfail - 1)->d_after : s.D[c];
            st = ST_BLOCKED;
            partner = (int32_t)holder;
        } else {
            al = s.rp_aloc[c];
            id = s.rp_ci[c];
            tc = s.rp_tc[c];
            D = s.rp_D[c];
            if (lost >= 0) {
                st = ST_BLOCKED;
                partner = (int32_t)holder;
            } else if (end == RP_END_NONSTATIC) {
                st = ST_BLOCKED;
                partner = s.rp_partner[c];
            } else {
                st = end == RP_END_STALL ? ST_STALLED : ST_RUNNING;
            }
        }
        s.aloc[c] = al;
        s.ci[c] = id;
        s.tc[c] = tc;
        s.D[c] = D;
        s.status[c] = st;
        s.nrec[c] = nrec0 + sfail;
        s.nlift[c] += pub_lifts;
        if (st == ST_BLOCKED) {
            s.partner[c] = partner;
            s.vt[c] = fmax(tc, tw);
            note_blocked(s, c, partner);
        } else {
            s.vt[c] = INFINITY;
        }
        if (over) {
            atomicAdd(s.lc + LC_WEAK, 1ull);
            atomicAdd(s.lc + LC_WWEAK, 1ull);
        }
        atomicAdd(s.lc + LC_P1LIFTS, (unsigned long long)pub_lifts);
    }
    (void)blocked;
    __syncwarp();
}

// ------------------------------------------------- continuation in a row

// Outcome of row_cont_member.
enum { RC_GENERAL = 0, RC_DONE = 1, RC_FAIL = 2, RC_NONSTATIC = 3 };

// Continues member c of a repair component (the first repair round,
// continue_component) along its row with the window of the row pass, for as
// long as the general step would do nothing else: the member's disk and each
// next one have both neighbour rows out of reach, and every cell the scan
// covers is held by a member of the component (so no claim is needed and the
// cells change only in this warp). The step follows scan_step in CONT mode:
// the scan runs to D, and the horizon condition (Eq. 2) must hold for every
// scanned corridor disk -- certified, for a disk with t_j != 0, by RN(t_i +
// (dx - d)) > t_j, which bounds RN(t_i + tau) from below; the winner and
// everything in doubt are evaluated exactly (rp_exact). Events are written at
// once, as commit_step writes them. Returns RC_DONE (stalled or paused; st is
// set), RC_FAIL, RC_NONSTATIC (*ns_owner: another chain's disk in reach) or
// RC_GENERAL: the general step takes over from the state in r. members: the
// component's members, one per lane (nmem <= 32).
template <int C>
__device__ int row_cont_member(const Dev &s, int c, int round, ChainReg &r, int32_t &nrec,
                               uint32_t &cnt, double tw, double tend, int nmem, int my_member,
                               int &st, uint32_t *ns_owner) {
    constexpr int G = 32 / C;
    const int lane = threadIdx.x & 31, gme = lane / C;
    const StopK sk = stopk_of(s);
    const double dd = s.d, LL = s.L;
    const int cap = s.cap, nc = s.nc;
    RowChain ch;
    ch.c = c;
    const uint32_t cell0 = r.iloc / C;
    ch.row = (int)(cell0 / (uint32_t)nc);
    ch.u0 = (int)(cell0 % (uint32_t)nc);
    ch.wbase = 0;
    ch.gbase = 0;
    ch.i = r.i;
    ch.xi = r.xi;
    ch.yi = r.yi;
    ch.ti = r.ti;
    ch.D = r.D;
    ch.front = -1;
    ch.li = (int)(r.iloc % C);
    ch.iskp = RP_SKIP_ALL;
    RowLane w;
    int hold = -1;     // the chain holding this lane's cell (strongly), -1 none
    bool cok = false;  // ... and it is a member
    auto load = [&](int pos) {  // (lanes may diverge: no shuffle)
        rp_load<C>(s, ch, w, pos);
        int col = ch.u0 + ch.wbase + pos;
        if (col >= nc) col -= nc;
        const uint32_t cw = __ldcg(s.claim + (uint32_t)ch.row * (uint32_t)nc + (uint32_t)col);
        hold = (cw == 0u || (cw & CLAIM_WEAK)) ? -1 : (int)(cw - 1u);
    };
    auto members = [&]() {  // (uniform)
        bool mem = false;
        for (int q = 0; q < nmem; ++q) mem |= __shfl_sync(FULL, my_member, q) == hold;
        cok = hold >= 0 && mem;
    };
    load(gme);
    rp_prefetch<C>(s, ch, G);
    members();
    int vi = 0;
    ch.fx = __dsub_rn(ch.xi, __shfl_sync(FULL, w.colx, ch.li));
    // this lane's step decided ahead where D does not enter (rc_prep)
    double ptau, pxn, pfx;
    int pR;
    unsigned nsR, cokm;
    uint32_t pinfo;
    float pthr[3], pxf, ptf;
    auto links = [&]() {
        int nxr, rnk;
        rp_links<C>(s, ch, w, &nxr, &rnk);
        rc_prep<C>(s, ch, w, nxr, rnk, ptau, pxn, pfx, pR, nsR, pinfo, pthr, pxf, ptf);
        cokm = __ballot_sync(FULL, cok);
    };
    links();
    int nx = __shfl_sync(FULL, w.nx, ch.li);
    double bnx = __shfl_sync(FULL, w.b, ch.li);
    auto v_of_lane = [&](int l) { return ((l / C) - ch.gbase) & (G - 1); };
    // the window slides when a step's scan to D would leave it (or the
    // active column reaches G - 2)
    bool need_slide = false;
    for (;;) {
        if (vi >= G - 2 || (need_slide && vi > 0)) {
            need_slide = false;
            if (ch.wbase + vi + G > nc) return RC_GENERAL;
            const int v0 = (gme - ch.gbase) & (G - 1);
            const int h = vi;
            ch.wbase += h;
            ch.gbase = (ch.gbase + h) & (G - 1);
            if (v0 < h) load(v0 + G - h);
            rp_prefetch<C>(s, ch, ch.wbase + G);
            members();
            vi = 0;
            links();
            nx = __shfl_sync(FULL, w.nx, ch.li);
            bnx = __shfl_sync(FULL, w.b, ch.li);
        }
        const int v = (gme - ch.gbase) & (G - 1);
        // a batch of steps that lift within their slots: per step in uniform
        // registers the scan to D (its columns all held by members, no other
        // chain's disk after the active one in them, the candidate after the
        // target above tau), Eq. 2 on every scanned disk with t_j != 0 (lane
        // by lane), t_i + tau and D - tau; then each step's record and cell
        // writes by the lane of the disk that moved, all at once. What the
        // batch cannot decide is left to the step below.
        {
            int lk = ch.li, K = 0;
            double t = ch.ti, D = ch.D;
            bool pause = false;
            int my_k = -1;
            double my_t = 0.0, my_tn = 0.0, my_dn = 0.0;
            for (;;) {
                const uint32_t ci = __shfl_sync(FULL, pinfo, lk);
                if (!(ci & RC_PREP_OK)) break;
                const int vk = v_of_lane(lk);
                if (K > 0 && vk >= G - 2) break;
                if (nrec + K >= cap) break;
                const double tau = __shfl_sync(FULL, ptau, lk);
                if (!(dbits(tau) < dbits(D))) break;  // a stall: the step below
                // the scan to D: its columns, from the active disk's FP32 image
                // of thr(m) against trunc(D) + eps (decided where the images
                // lie farther apart than their error bound; else the step
                // below decides in FP64)
                int mst = 0;
                {
                    const float limk = __fadd_rn(d2f_trunc(D), sk.epsf);
                    bool doubt = !(sk.stop_e > 0.f);
#pragma unroll
                    for (int m = 1; m <= 3; ++m) {
                        const float dfm = __fsub_rn(__shfl_sync(FULL, pthr[m - 1], lk), limk);
                        if (mst == 0 && m < G - vk) {
                            if (dfm > sk.stop_e)
                                mst = m;
                            else if (!(dfm < -sk.stop_e))
                                doubt = true;
                        }
                    }
                    if (doubt || mst == 0) {
                        need_slide = mst == 0 && !doubt && vk > 0;
                        break;
                    }
                }
                const int pp = (int)(ci & 31u);
                if (v_of_lane(pp) - vk >= mst) break;
                // the scanned columns' lanes: mst groups from the active one's
                const int gs = ((ch.gbase + vk) & (G - 1)) * C, nb = mst * C;
                const unsigned run = nb >= 32 ? ~0u : ((1u << nb) - 1u);
                const unsigned sm = gs == 0 ? run : ((run << gs) | (run >> (32 - gs)));
                if (sm & ~cokm) break;
                const int Rk = __shfl_sync(FULL, pR, lk);
                {
                    const int lim = (vk + mst) * C;
                    const unsigned inrange = lim >= 32 ? ~0u : ((1u << lim) - 1u);
                    const unsigned after = Rk >= 31 ? 0u : ~((2u << Rk) - 1u);
                    if (nsR & inrange & after) break;
                }
                if ((int)((ci >> 8) & 31u) < vk + mst && !(ci & RC_PREP_NX2OK)) break;
                const double tn = __dadd_rn(t, tau);
                // Eq. 2 on the scanned disks with t_j != 0: the target by its
                // tau (t_i + tau is the step's new time), the others from the
                // FP32 image of t_i + (x_j - x_i - d) - t_j, decided where it lies
                // above the image's error bound, else in FP64
                const bool cz = w.id != EMPTY && pR > Rk && v < vk + mst && dbits(w.t) != 0ull;
                if (__any_sync(FULL, cz)) {
                    const float xkf = __shfl_sync(FULL, pxf, lk);
                    const float tkf = d2f_trunc(t);
                    bool bad = false, doubt = false;
                    if (cz) {
                        if (lane == pp) {
                            bad = !(dbits(tn) > dbits(w.t));
                        } else {
                            const float sbf = __fsub_rn(__fsub_rn(pxf, xkf), sk.df);
                            const float mf = __fsub_rn(__fadd_rn(tkf, sbf), ptf);
                            doubt = !(sbf > sk.stop_e && mf > sk.stop_e);
                        }
                    }
                    if (__any_sync(FULL, doubt)) {
                        const double xk = __shfl_sync(FULL, w.x, lk);
                        if (doubt) {
                            double dx = __dsub_rn(w.x, xk);
                            if (dneg(dx) && v > vk) dx = rp_add(dx, LL);
                            const double sb = __dsub_rn(dx, dd);
                            bad = dneg(sb) || !(dbits(__dadd_rn(t, sb)) > dbits(w.t));
                        }
                    }
                    if (__any_sync(FULL, bad)) break;
                }
                if (!(dbits(tn) < dbits(tend))) {  // pauses at the window end
                    pause = true;
                    break;
                }
                if (dbits(tn) < dbits(tw)) break;
                const double dn = __dsub_rn(D, tau);
                if (lane == lk) {
                    my_k = K;
                    my_t = t;
                    my_tn = tn;
                    my_dn = dn;
                }
                t = tn;
                D = dn;
                ++K;
                lk = pp;
            }
            if (K > 0) {
                const int nxl = w.nx;
                const int srcp = my_k >= 0 ? nxl : lane;
                const double xp = __shfl_sync(FULL, w.x, srcp);
                const double tp = __shfl_sync(FULL, w.t, srcp);
                const uint32_t idp = __shfl_sync(FULL, w.id, srcp);
                if (my_k >= 0) {
                    const uint32_t from = rp_loc_of<C>(s, ch, lane);
                    const uint32_t jloc = rp_loc_of<C>(s, ch, nxl);
                    const uint32_t seq = ((uint32_t)round << 24) | (cnt + (uint32_t)my_k);
                    ulonglong2 *q = (ulonglong2 *)rec_at(s, c, nrec + my_k);
                    q[0] = make_ulonglong2((unsigned long long)w.id | ((unsigned long long)from << 32),
                                           (unsigned long long)from | ((unsigned long long)idp << 32));
                    q[1] = make_ulonglong2((unsigned long long)jloc | ((unsigned long long)seq << 32),
                                           0ull);
                    q[2] = make_ulonglong2(dbits(w.x), dbits(my_t));
                    q[3] = make_ulonglong2(dbits(tp), dbits(my_tn));
                    q[4] = make_ulonglong2(dbits(ptau), dbits(pxn));
                    q[5] = make_ulonglong2(dbits(xp), dbits(my_dn));
                    // the disk moved within its slot and is static now
                    s.cx[from] = pxn;
                    s.ct[from] = my_tn;
                    s.cown[from] = OWN_STATIC;
                    w.x = pxn;
                    w.t = my_tn;
                    w.own = OWN_STATIC;
                    w.nx = -1;
                    w.bok = 0;
                } else if (lane == lk) {
                    const uint32_t al = rp_loc_of<C>(s, ch, lane);
                    s.cown[al] = OWN_ACTIVE | (uint32_t)c;
                    s.ct[al] = t;
                    w.t = t;
                    w.own = OWN_ACTIVE | (uint32_t)c;
                }
                if (lane == 0) {
                    s.nrec[c] = nrec + K;
                    atomicAdd(s.nlift + c, K);
                }
                __syncwarp();
                nrec += K;
                cnt += (uint32_t)K;
                ch.li = lk;
                ch.i = __shfl_sync(FULL, w.id, lk);
                ch.xi = __shfl_sync(FULL, w.x, lk);
                ch.yi = __shfl_sync(FULL, w.y, lk);
                ch.ti = t;
                ch.D = D;
                ch.fx = __shfl_sync(FULL, pfx, lk);
                vi = v_of_lane(lk);
                nx = __shfl_sync(FULL, w.nx, lk);
                bnx = __shfl_sync(FULL, w.b, lk);
                r.iloc = rp_loc_of<C>(s, ch, lk);
                r.i = ch.i;
                r.xi = ch.xi;
                r.yi = ch.yi;
                r.ti = t;
                r.D = D;
                r.skip = __shfl_sync(FULL, w.skp, lk);
            }
            if (pause) {
                st = ST_RUNNING;
                return RC_DONE;
            }
            if (K > 0) continue;
        }
        const float fxf = d2f_trunc(ch.fx);
        const bool occ = w.id != EMPTY;
        // the scan runs to D: its columns
        const unsigned smask = rp_stop_mask(sk, ch.fx, fxf, dbits(ch.D), G - vi);
        const unsigned above = smask & ~1u;
        const int mstop = above ? __ffs(above) - 1 : G - vi;
        if (mstop >= G - vi) {
            if (vi > 0) {  // slide first
                need_slide = true;
                continue;
            }
            return RC_GENERAL;
        }
        const bool scanned = v >= vi && v < vi + mstop;
        if (__any_sync(FULL, scanned && !cok)) return RC_GENERAL;
        const int pp = nx;
        double dx = __dsub_rn(w.x, ch.xi);
        const bool neg = dneg(dx);
        const bool wl = occ && neg && v > vi;
        if (__any_sync(FULL, wl) && wl) dx = rp_add(dx, LL);
        const double sub = __dsub_rn(dx, lane == pp ? bnx : dd);
        double taup = INFINITY;
        if (pp >= 0) {
            taup = __shfl_sync(FULL, sub, pp);
            if (dneg(taup)) taup = 0.0;
        }
        const bool lift = pp >= 0 && dbits(taup) < dbits(ch.D);
        const unsigned long long cur = lift ? dbits(taup) : dbits(ch.D);
        const bool cnd = occ && scanned && w.id != ch.i && !(neg && v == vi);
        bool bad = cnd && !(lift && lane == pp) &&
                   (w.own != OWN_STATIC || dneg(sub) ||
                    (lift ? !(dbits(sub) > cur) : !(dbits(sub) >= cur)));
        if (lift && lane == pp && w.own != OWN_STATIC) bad = true;
        // Eq. 2 on every scanned disk with t_j != 0, from the lower bound
        // (for the target its exact tau): RN(t_i + sub) > t_j
        const bool tz = cnd && dbits(w.t) != 0ull;
        if (__any_sync(FULL, tz) && tz) {
            if (dneg(sub) || !(dbits(__dadd_rn(ch.ti, sub)) > dbits(w.t))) bad = true;
        }
        RowStep rs;
        if (__any_sync(FULL, bad) || (lift && (((pp / C) - ch.gbase) & (G - 1)) - vi >= mstop)) {
            rs = rp_exact<C, true>(s, sk, ch, w, vi, fxf);
            if (rs.overflow || rs.mstop != mstop) return RC_GENERAL;
            if (rs.viol) return RC_FAIL;
            if (rs.nonstatic) {
                *ns_owner = rs.ns_owner;
                return RC_NONSTATIC;
            }
        } else {
            rs.lift = lift;
            rs.p = lift ? pp : -1;
            rs.tau = lift ? taup : ch.D;
        }
        // t_i + tau, x_i + tau, D - tau and the target's offset in its cell
        const int p = rs.p;
        const int pe = p >= 0 ? p : 0;
        const int a0 = (pe + 1) & 31, a1 = (pe + 2) & 31, a2 = (pe + 3) & 31;
        double opa = ch.D, opb = -rs.tau;
        if (lane == a0) {
            opa = ch.ti;
            opb = rs.tau;
        } else if (lane == a1) {
            opa = ch.xi;
            opb = rs.tau;
        } else if (p >= 0 && lane == p) {
            opa = w.x;
            opb = -w.colx;
        }
        const double sum = __dadd_rn(opa, opb);
        const double tnew = __shfl_sync(FULL, sum, a0);
        double xnew = __shfl_sync(FULL, sum, a1);
        if (!(dbits(tnew) < dbits(tend))) {  // pauses at the window end
            st = ST_RUNNING;
            return RC_DONE;
        }
        if (dbits(tnew) < dbits(tw)) return RC_FAIL;
        if (nrec >= cap) {
            if (lane == 0) atomicAdd(s.lc + LC_ERR_REC, 1ull);
            return RC_FAIL;
        }
        if (dbits(xnew) >= dbits(LL)) xnew = rp_sub(xnew, LL);
        const unsigned long long xb = dbits(xnew);
        const unsigned hm =
            __ballot_sync(FULL, lane % C == 0 && v >= vi && xb >= w.xlo && xb < w.xhi);
        if (!hm) return RC_GENERAL;
        const int gn = (__ffs(hm) - 1) / C;
        int ln = ch.li;
        if (gn != ch.li / C) {
            const unsigned em =
                __ballot_sync(FULL, w.id == EMPTY) & (((1u << C) - 1u) << (gn * C));
            if (!em) {
                if (lane == 0) atomicAdd(s.lc + LC_ERR_CAP, 1ull);
                return RC_FAIL;
            }
            ln = __ffs(em) - 1;
        }
        const uint32_t from = rp_loc_of<C>(s, ch, ch.li);
        const uint32_t to = rp_loc_of<C>(s, ch, ln);
        const uint32_t jloc = rs.lift ? rp_loc_of<C>(s, ch, p) : 0u;
        const double dnew = rs.lift ? __shfl_sync(FULL, sum, a2) : 0.0;
        const uint32_t own_i = rs.lift ? OWN_STATIC : (OWN_STALLED | (uint32_t)c);
        const uint32_t seq = ((uint32_t)round << 24) | cnt;
        // the event, written as commit_step writes it; the record by the
        // target's lane (its fields) and lane 0
        {
            ulonglong2 *q = (ulonglong2 *)rec_at(s, c, nrec);
            const bool tl = rs.lift ? lane == p : lane == 0;
            if (tl) {
                const uint32_t jid = rs.lift ? w.id : NONE;
                q[0] = make_ulonglong2((unsigned long long)ch.i | ((unsigned long long)from << 32),
                                       (unsigned long long)to | ((unsigned long long)jid << 32));
                q[3] = make_ulonglong2(rs.lift ? dbits(w.t) : 0ull, dbits(tnew));
                q[5] = make_ulonglong2(rs.lift ? dbits(w.x) : 0ull, dbits(dnew));
                if (rs.lift) {
                    s.cown[jloc] = OWN_ACTIVE | (uint32_t)c;
                    s.ct[jloc] = tnew;
                }
            }
            if (lane == 0) {
                q[1] = make_ulonglong2((unsigned long long)jloc | ((unsigned long long)seq << 32),
                                       0ull);
                q[2] = make_ulonglong2(dbits(ch.xi), dbits(ch.ti));
                q[4] = make_ulonglong2(dbits(rs.tau), dbits(xnew));
                if (to != from) {
                    s.cx[to] = xnew;
                    s.cy[to] = ch.yi;
                    s.cskp[to] = (uint8_t)RP_SKIP_ALL;
                    s.ct[to] = tnew;
                    s.cown[to] = own_i;
                    s.cid[to] = ch.i;
                    s.cid[from] = EMPTY;
                } else {
                    s.cx[from] = xnew;
                    s.ct[from] = tnew;
                    s.cown[from] = own_i;
                }
                s.nrec[c] = nrec + 1;
                if (rs.lift) atomicAdd(s.nlift + c, 1);
            }
        }
        ++nrec;
        ++cnt;
        double xj = 0.0, yj = 0.0, fxn = 0.0;
        uint32_t jid = NONE;
        if (rs.lift) {
            xj = __shfl_sync(FULL, w.x, p);
            yj = __shfl_sync(FULL, w.y, p);
            jid = __shfl_sync(FULL, w.id, p);
            fxn = __shfl_sync(FULL, sum, p);
            if (lane == p) {
                w.t = tnew;
                w.own = OWN_ACTIVE | (uint32_t)c;
            }
        }
        if (ln != ch.li && lane == ch.li) w.id = EMPTY;
        if (lane == ln) {
            w.id = ch.i;
            w.x = xnew;
            w.y = ch.yi;
            w.t = tnew;
            w.own = own_i;
            w.skp = RP_SKIP_ALL;
            w.nx = -1;
            w.bok = 0;
        }
        if (!rs.lift) {  // stalled
            r.iloc = to;
            r.xi = xnew;
            r.ti = tnew;
            r.D = 0.0;
            st = ST_STALLED;
            return RC_DONE;
        }
        const bool next_ok = !__ballot_sync(FULL, lane == p && w.skp != RP_SKIP_ALL);
        r.iloc = jloc;
        r.i = jid;
        r.xi = xj;
        r.yi = yj;
        r.ti = tnew;
        r.D = dnew;
        r.skip = __shfl_sync(FULL, w.skp, p);
        if (!next_ok) return RC_GENERAL;
        nx = __shfl_sync(FULL, w.nx, p);
        bnx = __shfl_sync(FULL, w.b, p);
        ch.i = jid;
        ch.li = p;
        vi = (((p / C) - ch.gbase) & (G - 1));
        ch.xi = xj;
        ch.yi = yj;
        ch.ti = tnew;
        ch.D = dnew;
        ch.fx = fxn;
    }
}

