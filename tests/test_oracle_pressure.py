"""Hard-disk pressure from the oracle's lifting statistics against an
independent Metropolis run (the equation of state pins the whole event loop:
a wrong contact distance, sign or periodic image moves the pressure).

ECMC estimator (one chain of length ell per leg, direction alternating +x/+y
between legs, start disk drawn uniformly at each breakpoint):
    beta P / rho = 1 + sum over liftings of (x_j - x_i) / total chain length.
Metropolis (tests/metropolis.c): the 2D virial contact value
    beta P / rho = 1 + (pi/2) d^2 (N-1)/A g(d+),
with g normalised to the N-1 other disks and extrapolated to contact.
Both at N = 32, eta = 0.40 in the same periodic box; they must agree within
four combined standard errors (block averages).
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def metro():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    lib = os.path.join(out, "libmetropolis.so")
    src = os.path.join(HERE, "metropolis.c")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, lib)
    m = C.CDLL(lib)
    m.metro_run.restype = C.c_double
    return m


def metropolis_pressure(metro, start, blocks=10, sweeps=20000, every=2, nb=20, dr=0.005):
    n, L, d = start.n, start.box, start.d
    x, y = start.x.copy(), start.y.copy()
    dp = C.POINTER(C.c_double)
    r = d + (np.arange(nb) + 0.5) * dr
    shell = np.pi * ((d + (np.arange(nb) + 1) * dr) ** 2 - (d + np.arange(nb) * dr) ** 2)
    est = []
    for b in range(blocks):
        hist = np.zeros(nb)
        metro.metro_run(n, C.c_double(L), C.c_double(d), x.ctypes.data_as(dp),
                        y.ctypes.data_as(dp), C.c_double(0.3), 2000 if b == 0 else 0,
                        sweeps, every, nb, C.c_double(dr), hist.ctypes.data_as(dp),
                        C.c_uint64(1000 + b))
        g = hist / (sweeps // every) / (n * (n - 1) / 2 * shell / L ** 2)
        g0 = np.polyval(np.polyfit(r, g, 2), d)
        est.append(1 + np.pi / 2 * d * d * (n - 1) / L ** 2 * g0)
    return np.mean(est), np.std(est) / np.sqrt(blocks)


def ecmc_pressure(start, blocks=10, legs=2000, seed=3):
    n, L = start.n, start.box
    rng = np.random.default_rng(seed)
    x, y = start.x.copy(), start.y.copy()
    ell = 0.5 * L
    est = []
    for _ in range(blocks):
        jumps, length = 0.0, 0.0
        for leg in range(legs):
            act = rng.choice(n, 1).astype(np.int32)
            if leg % 2 == 0:
                r = O.run_leg(x, y, act, L, ell, search=0)
                x = r.x
            else:  # +y: the same oracle on exchanged coordinates
                r = O.run_leg(y, x, act, L, ell, search=0)
                y = r.x
            jumps += float(np.sum((r.log["xj"] - r.log["xi"]) % L))
            length += ell
        est.append(1 + jumps / length)
    return np.mean(est), np.std(est) / np.sqrt(blocks)


def test_ecmc_pressure_matches_metropolis(metro):
    start = synth.rsa_start(32, 0.40, 1, seed=5)
    pm, sm = metropolis_pressure(metro, start)
    pe, se = ecmc_pressure(start)
    assert 2.5 < pm < 3.1  # near the hard-disk equation of state at eta = 0.4
    assert abs(pe - pm) < 4 * np.hypot(sm, se), (pe, se, pm, sm)
