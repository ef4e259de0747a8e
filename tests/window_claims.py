"""Claim windows checked one by one, independently of the oracle's C code.

A leg of length ell is cut into W claim windows of global time,
[w ell/W, (w+1) ell/W). For each window this module rebuilds the state at its
start from a lifting log (every lifting i -> j sets x_i to the contact
position and t_i = t_j to the event time, Eq. 1; the chain's remaining length
drops by tau), runs every chain alone from there through its events before
the window's end -- the other disks static, the step taken over all disks
(Sec. 2.2, Eq. 2's time of flight), the cells the cell scan reads derived
from its stop rule -- and compares the claim sets. Written in numpy from the
readings stated below, not from the oracle's source:

- tau_ij = dx - sqrt(d^2 - dy^2) (0 if negative) with dx the forward image
  of x_j - x_i (+L if negative), dy the minimum image, j a candidate iff
  |dy| < d; a disk j with t_i + tau < t_j is one lap away (tau + L); the
  argmin of (tau, j) lifts iff tau < D, else the chain moves by D and stalls.
- Cells: side a = L / nc, coordinate int(v nc / L) clamped to nc - 1. A step
  of disk i in cell (cx, cy) reads rows cy-1 .. cy+1 and columns cx + m,
  m = 0, 1, ...; before column m >= 1 it stops when
  (m a - (x_i - cx a)) - d > min(best so far, D) + L 2^-30.
- The window's flag is 1 iff two chains' claim sets share a cell.
"""
from __future__ import annotations

import math

import numpy as np


class Geometry:
    def __init__(self, L: float, d: float, nc: int):
        self.L, self.d, self.nc = float(L), float(d), int(nc)
        self.a = self.L / self.nc
        self.inv_a = self.nc / self.L
        self.eps = math.ldexp(self.L, -30)

    def coord(self, v):
        c = np.floor(np.asarray(v) * self.inv_a).astype(np.int64)
        return np.clip(c, 0, self.nc - 1)


def window_end(ell: float, W: int, w: int) -> float:
    return math.inf if w + 1 >= W else (float(w + 1) * ell) / float(W)


def replay(x0, active0, ell, log, t_cut):
    """State after the liftings with event time < t_cut: x, t, active, D.
    The log lists a leg's liftings in global-time order."""
    x = np.array(x0, dtype=np.float64, copy=True)
    t = np.zeros_like(x)
    act = np.array(active0, dtype=np.int64, copy=True)
    D = np.full(len(act), float(ell))
    for e in log:
        if not e["t"] < t_cut:
            break
        c, i, j = int(e["c"]), int(e["i"]), int(e["j"])
        assert act[c] == i
        x[i] = e["xi"]
        t[i] = e["t"]
        t[j] = e["t"]
        D[c] = D[c] - e["tau"]
        act[c] = j
    return x, t, act, D


def taus(g: Geometry, x, y, t, i):
    """Time of flight of i towards every disk (inf outside the corridor or
    for i itself), in i's lazily advanced frame."""
    a = np.abs(y - y[i])
    a = np.where(g.L - a < a, g.L - a, a)
    inside = a < g.d
    b = np.sqrt(np.where(inside, g.d * g.d - a * a, 0.0))
    dx = x - x[i]
    dx = np.where(dx < 0.0, dx + g.L, dx)
    tau = dx - b
    tau = np.where(tau < 0.0, 0.0, tau)
    tau = np.where(inside, tau, np.inf)
    tau[i] = np.inf
    lap = np.isfinite(tau) & (t[i] + tau < t)
    return np.where(lap, tau + g.L, tau)


def step(g: Geometry, x, y, t, i, D):
    """One step of disk i with remaining length D: (lift, j, tau, cells read)."""
    tau = taus(g, x, y, t, i)
    fin = np.flatnonzero(np.isfinite(tau))
    if fin.size:
        best = fin[np.lexsort((fin, tau[fin]))[0]]
        btau, bj = float(tau[best]), int(best)
    else:
        btau, bj = math.inf, -1
    cx, cy = int(g.coord(x[i])), int(g.coord(y[i]))
    fx = x[i] - float(cx) * g.a
    cols = (g.coord(x[fin]) - cx) % g.nc
    col_best = np.full(g.nc, np.inf)
    np.minimum.at(col_best, cols, tau[fin])
    cells = set()
    running = math.inf
    for m in range(g.nc):
        if m >= 1:
            lim = running if running < D else D
            if ((float(m) * g.a - fx) - g.d) > lim + g.eps:
                break
        col = (cx + m) % g.nc
        for r in (cy - 1, cy, cy + 1):
            cells.add((r % g.nc) * g.nc + col)
        running = min(running, col_best[m])
    if btau < D:
        return True, bj, btau, cells
    return False, -1, D, cells


def wrap_add(v, dv, L):
    r = v + dv
    return r - L if r >= L else r


def run_alone(g: Geometry, x, y, t, i, D, t_end):
    """Runs one chain alone on (x, t) in place through its events before
    t_end; returns (its claim set, active disk, remaining length)."""
    claims = set()
    while True:
        lift, j, tau, cells = step(g, x, y, t, i, D)
        claims |= cells
        if not (t[i] + tau < t_end):
            break
        tn = t[i] + tau
        x[i] = wrap_add(x[i], tau, g.L)
        if not lift:
            t[i] = tn
            D = 0.0
            break
        t[j] = tn
        t[i] = tn
        D = D - tau
        i = j
    return claims, i, D


def window_flags(g: Geometry, x0, y, active0, ell, W, log):
    """Per-window flags of a leg from its lifting log (global-time order)."""
    flags = []
    for w in range(W):
        t0 = 0.0 if w == 0 else window_end(ell, W, w - 1)
        x, t, act, D = replay(x0, active0, ell, log, t0)
        owner = {}
        hit = 0
        for c in range(len(act)):
            if not D[c] > 0.0:
                continue
            xs, ts = x.copy(), t.copy()
            claims, _, _ = run_alone(g, xs, y, ts, int(act[c]), float(D[c]),
                                     window_end(ell, W, w))
            for q in claims:
                if owner.setdefault(q, c) != c:
                    hit = 1
        flags.append(hit)
    return flags


def compose_window(g: Geometry, x0, y, active0, ell, W, log, w):
    """Lemma 2 for window w: every chain run alone through the window, one
    after another in chain order on the shared state, from the window-start
    state. Returns (x, t, active)."""
    t0 = 0.0 if w == 0 else window_end(ell, W, w - 1)
    x, t, act, D = replay(x0, active0, ell, log, t0)
    for c in range(len(act)):
        if not D[c] > 0.0:
            continue
        _, i, _ = run_alone(g, x, y, t, int(act[c]), float(D[c]), window_end(ell, W, w))
        act[c] = i
    return x, t, act
