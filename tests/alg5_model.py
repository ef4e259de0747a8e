"""State-space exploration of a sequential-consistency model of Alg. 5.

Each thread (one chain) is a small program whose every step is ONE access
to shared memory -- a read of a disk's x or local time, the compare-and-swap
of a tag, or one write -- with the thread-local arithmetic attached to the
access that feeds it. A switch may pick any thread at any step. Following the
proof of Lemma 3, all states reachable from the initial state are
enumerated; the absorbing states are "terminate" (every thread has stalled
at the breakpoint) and "abort" (a thread saw the horizon condition, Eq. 2,
fail). The oracle is pinned by requiring every terminate state to equal its
global-time result.

What a thread does, written from the method's meaning (Sec. 2.2-2.3) with
the readings used throughout (tau = forward dx - b, minimum image in y,
strict corridor, x wrapped into [0, L)):
  scan      for every other disk q: read x_q (time of flight from the
            thread's own disk i), read t_q (horizon condition t_i + tau > t_q
            or abort; the least (tau, q) so far is kept, ties to the lower q);
  claim     if the best tau is below the remaining length D: compare-and-swap
            the target's tag from static to this chain (a failure restarts
            the scan), re-read x_j and release the tag if j moved since the
            scan (restart), else write t_j, t_i and x_i -- the local times
            before the position (Remark 11) -- and free i's tag; activity
            passes to j and D shrinks by tau;
  stall     otherwise write t_i + D, x_i + D and tag i as stalled.
``late_time`` writes x_i before t_i (the order Remark 11 warns against) for
the mutation test.
"""
from __future__ import annotations

import math
from collections import deque

INF = math.inf
STATIC, STALLED = 0, -1

# phases: the shared access a thread makes next
READ_X, READ_T, CAS, VERIFY, RELEASE, SET_TJ, SET_A, SET_B, FREE_I, \
    STALL_T, STALL_X, STALL_TAG, DONE = range(13)


def time_of_flight(xi, yi, xj, yj, L, d):
    a = abs(yj - yi)
    if L - a < a:
        a = L - a
    if not (a < d):
        return INF
    b = math.sqrt(d * d - a * a)
    dx = xj - xi
    if dx < 0.0:
        dx += L
    tau = dx - b
    if tau < 0.0:
        tau = 0.0
    return tau


def wrap_add(x, dx, L):
    r = x + dx
    if r >= L:
        r -= L
    return r


def _first(q, i, n):
    """The first candidate index >= q other than the active disk i (n: none)."""
    while q < n and q == i:
        q += 1
    return q


# thread locals: (phase, i, D, q, tau_q, x_q, bj, btau, bx)
def explore(x, y, active, L, ell, d=1.0, late_time=False, max_states=2_000_000):
    """Returns (terminal_states, n_states, aborted, all_reach_absorbing)."""
    n = len(x)
    k = len(active)
    tag0 = [STATIC] * n
    for c, a in enumerate(active):
        tag0[a] = c + 1

    def scan_start(i, D):
        q = _first(0, i, n)
        ph = READ_X if q < n else None
        return (ph, i, D, q, INF, 0.0, i, D, INF)

    def after_scan(th):
        ph, i, D, q, tq, xq, bj, btau, bx = th
        if btau < D:
            return (CAS, i, D, q, tq, xq, bj, btau, bx)
        return (STALL_T, i, D, q, tq, xq, bj, btau, bx)

    def start(i, D):
        th = scan_start(i, D)
        return th if th[0] is not None else after_scan(th)

    th0 = tuple(start(int(a), ell) for a in active)
    s0 = (tuple(float(v) for v in x), (0.0,) * n, tuple(tag0), th0)
    ABORT = ("abort",)
    first_write, second_write = (SET_B, SET_A) if late_time else (SET_A, SET_B)

    def step(state, c):
        xs, ts, tags, ths = state
        ph, i, D, q, tq, xq, bj, btau, bx = ths[c]
        if ph == DONE:
            return None
        xs, ts, tags = list(xs), list(ts), list(tags)
        me = c + 1
        if ph == READ_X:
            xq = xs[q]
            th = (READ_T, i, D, q, time_of_flight(xs[i], y[i], xq, y[q], L, d), xq, bj, btau, bx)
        elif ph == READ_T:
            if ts[i] + tq < ts[q]:
                return ABORT
            if tq < btau:
                bj, btau, bx = q, tq, xq
            q = _first(q + 1, i, n)
            th = (READ_X, i, D, q, INF, 0.0, bj, btau, bx)
            if q >= n:
                th = after_scan(th)
        elif ph == CAS:
            if tags[bj] == STATIC:
                tags[bj] = me
                th = (VERIFY, i, D, q, tq, xq, bj, btau, bx)
            else:
                th = start(i, D)
        elif ph == VERIFY:
            th = (SET_TJ if xs[bj] == bx else RELEASE, i, D, q, tq, xq, bj, btau, bx)
        elif ph == RELEASE:
            tags[bj] = STATIC
            th = start(i, D)
        elif ph == SET_TJ:
            ts[bj] = ts[i] + btau
            th = (first_write, i, D, q, tq, xq, bj, btau, bx)
        elif ph in (SET_A, SET_B):
            if ph == SET_A:
                ts[i] = ts[i] + btau
            else:
                xs[i] = wrap_add(xs[i], btau, L)
            nxt = second_write if ph == first_write else FREE_I
            th = (nxt, i, D, q, tq, xq, bj, btau, bx)
        elif ph == FREE_I:
            tags[i] = STATIC
            th = start(bj, D - btau)
        elif ph == STALL_T:
            ts[i] = ts[i] + D
            th = (STALL_X, i, D, q, tq, xq, bj, btau, bx)
        elif ph == STALL_X:
            xs[i] = wrap_add(xs[i], D, L)
            th = (STALL_TAG, i, D, q, tq, xq, bj, btau, bx)
        else:  # STALL_TAG
            tags[i] = STALLED
            th = (DONE, i, 0.0, 0, INF, 0.0, i, 0.0, INF)
        nth = list(ths)
        nth[c] = th
        return (tuple(xs), tuple(ts), tuple(tags), tuple(nth))

    index = {s0: 0}
    states = [s0]
    succ: list[list[int]] = []
    q = deque([0])
    aborted = False
    abort_id = None
    while q:
        u = q.popleft()
        su = states[u]
        out = []
        if su != ABORT:
            for c in range(k):
                v = step(su, c)
                if v is None:
                    continue
                if v == ABORT:
                    aborted = True
                if v not in index:
                    index[v] = len(states)
                    states.append(v)
                    q.append(index[v])
                    if len(states) > max_states:
                        raise RuntimeError("state space too large")
                out.append(index[v])
        succ.append(out)
    terminals = [s for s in states if s != ABORT and all(t[0] == DONE for t in s[3])]
    absorbing = {index[s] for s in terminals}
    if ABORT in index:
        abort_id = index[ABORT]
        absorbing.add(abort_id)
    # every state must reach an absorbing state (Lemma 3's absorbing chain)
    pred: list[list[int]] = [[] for _ in states]
    for u, outs in enumerate(succ):
        for v in outs:
            pred[v].append(u)
    reach = set(absorbing)
    dq = deque(absorbing)
    while dq:
        v = dq.popleft()
        for u in pred[v]:
            if u not in reach:
                reach.add(u)
                dq.append(u)
    return terminals, len(states), aborted, len(reach) == len(states)
