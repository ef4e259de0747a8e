"""State-space exploration of the sequential-consistency model of Alg. 5.

Each thread runs the statements of Alg. 5 (Sec. 2.3) one at a time; a switch
may pick any thread at any step. Following the proof of Lemma 3, all states
reachable from the initial state are enumerated; absorbing states are
"terminate" (every thread waits at statement 26) and "abort" (a horizon
violation, statement 5). The oracle is pinned by requiring every terminate
state to equal its global-time result.

The statements are written from the pseudo-code's meaning, with the readings
used throughout (tau = forward dx - b, minimum image in y, strict corridor,
x wrapped into [0, L)). ``swap_15_16`` exchanges statements 15 and 16
(Remark 11) for the mutation test.
"""
from __future__ import annotations

import math
from collections import deque

INF = math.inf
STATIC, STALLED = 0, -1


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


# thread locals: (pc, i, j, tau_t, x_t, dist, p, nbr, x_nbr, tau_in)
def explore(x, y, active, L, ell, d=1.0, swap_15_16=False, max_states=2_000_000):
    """Returns (terminal_states, n_states, aborted, all_reach_absorbing)."""
    n = len(x)
    k = len(active)
    tag0 = [STATIC] * n
    for c, a in enumerate(active):
        tag0[a] = c + 1
    th0 = tuple((1, int(a), int(a), ell, INF, ell, 0, -1, 0.0, 0.0) for a in active)
    s0 = (tuple(float(v) for v in x), (0.0,) * n, tuple(tag0), th0)
    ABORT = ("abort",)

    order15 = (16, 15) if swap_15_16 else (15, 16)

    def step(state, c):
        xs, ts, tags, ths = state
        pc, i, j, tau_t, x_t, dist, p, nbr, x_nbr, tau_in = ths[c]
        xs, ts, tags = list(xs), list(ts), list(tags)
        me = c + 1
        if pc == 26:
            return None
        if pc == 1:
            tau_t, j, x_t, p, pc = dist, i, INF, 0, 2
        elif pc == 2:
            q = p
            while q < n and q == i:
                q += 1
            if q < n:
                nbr, p, pc = q, q + 1, 3
            else:
                pc = 10
        elif pc == 3:
            x_nbr, pc = xs[nbr], 4
        elif pc == 4:
            tau_in, pc = time_of_flight(xs[i], y[i], x_nbr, y[nbr], L, d), 5
        elif pc == 5:
            if ts[i] + tau_in < ts[nbr]:
                return ABORT
            pc = 6
        elif pc == 6:
            pc = 7 if tau_in < tau_t else 2
        elif pc == 7:
            j, pc = nbr, 8
        elif pc == 8:
            x_t, pc = x_nbr, 9
        elif pc == 9:
            tau_t, pc = tau_in, 2
        elif pc == 10:
            if tags[j] == STATIC:
                tags[j] = me
            pc = 11
        elif pc == 11:
            pc = 12 if tags[j] == me else 1
        elif pc == 12:
            pc = 13 if tau_t < dist else 21
        elif pc == 13:
            pc = 14 if x_t == xs[j] else 20
        elif pc == 14:
            ts[j] = ts[i] + tau_t
            pc = order15[0]
        elif pc in (15, 16):
            if pc == 15:
                ts[i] = ts[i] + tau_t
            else:
                xs[i] = wrap_add(xs[i], tau_t, L)
            pc = order15[1] if pc == order15[0] else 17
        elif pc == 17:
            tags[i], pc = STATIC, 18
        elif pc == 18:
            dist, pc = dist - tau_t, 19
        elif pc == 19:
            i, pc = j, 25
        elif pc == 20:
            tags[j], pc = STATIC, 1
        elif pc == 21:
            ts[i], pc = ts[i] + tau_t, 22
        elif pc == 22:
            xs[i], pc = wrap_add(xs[i], tau_t, L), 23
        elif pc == 23:
            dist, pc = 0.0, 24
        elif pc == 24:
            tags[i], pc = STALLED, 25
        elif pc == 25:
            pc = 1 if dist > 0.0 else 26
        nth = list(ths)
        nth[c] = (pc, i, j, tau_t, x_t, dist, p, nbr, x_nbr, tau_in)
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
    terminals = [s for s in states if s != ABORT and all(t[0] == 26 for t in s[3])]
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
