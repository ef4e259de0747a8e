"""Seeded synthetic inputs: jittered square-lattice starts and start-disk draws.

This module only makes inputs. It holds none of the ECMC arithmetic, and both
the CUDA path and the CPU oracle receive the arrays it returns.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw number ``i`` (0-based) of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15 mod 2**64)``. A draw becomes a double
in [0, 1) from its top 53 bits.

Workload recipe (the hard-disk box of Sec. 1 of the paper):
  * N = M*M disks of diameter d in a periodic square box of side
    L = sqrt(N*pi*d*d / (4*eta)); lattice spacing s = L / M.
  * disk id = c*M + r sits at ((c + 1/2)*s + u1, (r + 1/2)*s + u2) with
    u = (2*U - 1) * jitter; draws are taken in site order, c-major, x then y.
  * k start disks are then drawn without replacement with Floyd's algorithm
    from the same stream, in the order Floyd inserts them (chain c starts on
    the c-th inserted disk).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_scalar(seed: int, i: int) -> int:
    """Draw ``i`` of stream ``seed`` as a Python int (reference for the vector form)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def to_unit(z: np.ndarray) -> np.ndarray:
    """Top 53 bits of each draw as a double in [0, 1)."""
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def box_side(n: int, eta: float, d: float = 1.0) -> float:
    """L with packing fraction eta = n*pi*d^2 / (4 L^2) (d = diameter)."""
    return math.sqrt(n * math.pi * d * d / (4.0 * eta))


@dataclass
class Start:
    """A lifted start configuration {C_h, A_h}: positions plus chain start disks."""

    x: np.ndarray  # float64 [n]
    y: np.ndarray  # float64 [n]
    active: np.ndarray  # int32 [k], chain c starts on disk active[c]
    box: float  # L
    d: float
    m: int  # lattice side (0 for non-lattice starts)
    seed: int

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def k(self) -> int:
        return int(self.active.shape[0])


def floyd_sample(seed: int, start: int, n: int, k: int) -> np.ndarray:
    """k distinct ids in [0, n), Floyd's algorithm, draws from ``start`` on."""
    if k > n:
        raise ValueError("k > n")
    draws = splitmix64(seed, start, k)
    chosen: list[int] = []
    seen: set[int] = set()
    for step, jj in enumerate(range(n - k, n)):
        z = int(draws[step])
        t = ((z >> 11) * (jj + 1)) >> 53  # uniform in [0, jj]
        pick = jj if t in seen else t
        seen.add(pick)
        chosen.append(pick)
    return np.asarray(chosen, dtype=np.int32)


def lattice_start(m: int, eta: float, k: int, seed: int, jitter: float = 0.01,
                  d: float = 1.0) -> Start:
    """Jittered M x M square lattice at packing fraction eta with k start disks."""
    n = m * m
    L = box_side(n, eta, d)
    s = L / m
    u = to_unit(splitmix64(seed, 0, 2 * n))
    ux = (2.0 * u[0::2] - 1.0) * jitter
    uy = (2.0 * u[1::2] - 1.0) * jitter
    c = np.repeat(np.arange(m, dtype=np.float64), m)  # id = c*m + r
    r = np.tile(np.arange(m, dtype=np.float64), m)
    x = (c + 0.5) * s + ux
    y = (r + 0.5) * s + uy
    active = floyd_sample(seed, 2 * n, n, k)
    return Start(x=x, y=y, active=active, box=L, d=d, m=m, seed=seed)


def staggered_start(m: int, eta: float, k: int, seed: int, row_shift: float = 0.2,
                    pair_shift: float = 0.0, jitter: float = 0.01,
                    d: float = 1.0) -> Start:
    """M x M lattice (M even) with every odd row moved by s/2 along x and row r
    moved along y by (-1)^r pair_shift plus its own uniform draw in
    [-row_shift, row_shift].

    Some adjacent rows then lie within d in y and exchange liftings, others
    lie farther apart (pair_shift > 0: rows 2p and 2p + 1 close, pairs far
    apart). Draws: the jitter as in ``lattice_start``, then one per row, then
    Floyd's start disks. At eta = 0.5 (s = 1.2533 d) total shifts up to
    0.21 d keep every pair of disks at least d apart.
    """
    assert m % 2 == 0
    n = m * m
    L = box_side(n, eta, d)
    s = L / m
    u = to_unit(splitmix64(seed, 0, 2 * n))
    ux = (2.0 * u[0::2] - 1.0) * jitter
    uy = (2.0 * u[1::2] - 1.0) * jitter
    shift = (2.0 * to_unit(splitmix64(seed, 2 * n, m)) - 1.0) * row_shift
    shift = shift + np.where(np.arange(m) % 2 == 0, pair_shift, -pair_shift)
    c = np.repeat(np.arange(m, dtype=np.float64), m)  # id = c*m + r
    ri = np.tile(np.arange(m), m)
    x = np.mod((c + 0.5 + 0.5 * (ri % 2)) * s + ux, L)
    y = np.mod((ri + 0.5) * s + shift[ri] + uy, L)
    active = floyd_sample(seed, 2 * n + m, n, k)
    return Start(x=x, y=y, active=active, box=L, d=d, m=m, seed=seed)


def rsa_start(n: int, eta: float, k: int, seed: int, d: float = 1.0,
              max_tries: int = 10_000_000) -> Start:
    """Random sequential addition of n disks (non-lattice test starts, eta <~ 0.5).

    Candidate centres are uniform in the box; a candidate overlapping an
    accepted disk (periodic distance < d) is rejected. The k start disks are
    drawn with Floyd's algorithm after the last accepted disk.
    """
    L = box_side(n, eta, d)
    xs: list[float] = []
    ys: list[float] = []
    draw = 0
    while len(xs) < n:
        if draw // 2 > max_tries:
            raise RuntimeError("RSA did not converge; lower eta")
        z = splitmix64(seed, draw, 2)
        draw += 2
        cx = float(to_unit(z[:1])[0]) * L
        cy = float(to_unit(z[1:])[0]) * L
        ok = True
        for px, py in zip(xs, ys):
            dx = abs(px - cx)
            dx = min(dx, L - dx)
            dy = abs(py - cy)
            dy = min(dy, L - dy)
            if dx * dx + dy * dy < d * d:
                ok = False
                break
        if ok:
            xs.append(cx)
            ys.append(cy)
    active = floyd_sample(seed, draw, n, k)
    return Start(x=np.asarray(xs), y=np.asarray(ys), active=active, box=L, d=d,
                 m=0, seed=seed)


def lattice_m_for(n_target: int) -> int:
    """Lattice side for a requested disk count: M = round(sqrt(n)), N := M*M."""
    return max(2, int(round(math.sqrt(n_target))))
