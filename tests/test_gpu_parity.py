"""GPU path (libecmc through its C-ABI) against the CPU oracle.

Tolerance: bit-exact. Both sides evaluate the same IEEE-754 double operations
in the same order (no FMA contraction, correctly rounded sqrt), so positions,
local times, liftings (Eq. 1: i, j, t, tau, x, x') and the per-leg conflict
flags must agree exactly; the positions bar of 1e-12 d is met with zero error.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import ecmc, synth

pytestmark = pytest.mark.gpu


def run_gpu(start, ell, n_legs, nc=0, log=True, undo_cap=0, windows=1):
    sysm = ecmc.System(start.x, start.y, start.active, start.box, ell, d=start.d,
                       cells_per_side=nc, log=log, undo_cap=undo_cap,
                       log_cap=max(1 << 16, 64 * start.k * n_legs * 64), windows=windows)
    flags, done = sysm.run(n_legs)
    assert done == n_legs
    x, y, t, a = sysm.positions()
    logs = sysm.liftings() if log else None
    st = sysm.stats()
    sysm.close()
    return flags, x, y, t, a, logs, st


def run_oracle(start, ell, n_legs, nc=0, windows=1):
    ncell = nc or O.default_cells(start.box, start.d)
    last, legs = O.run_legs(start.x, start.y, start.active, start.box, ell, n_legs,
                            d=start.d, nc=ncell, windows=windows)
    flags = np.array([r.flag for r in legs], dtype=np.uint8)
    log = np.concatenate([r.log for r in legs]) if legs else np.zeros(0, O.LIFT_DTYPE)
    last.window_flags = int(sum(int(r.wflags.sum()) for r in legs))
    return flags, last, log


def chain_order(log):
    """Lifting records grouped leg by leg, chain by chain, each chain's in order."""
    idx = np.lexsort((np.arange(len(log)), log["c"], log["leg"]))
    return log[idx]


def assert_parity(start, ell, n_legs, nc=0, windows=1):
    gf, gx, gy, gt, ga, glog, st = run_gpu(start, ell, n_legs, nc, windows=windows)
    of, last, olog = run_oracle(start, ell, n_legs, nc, windows=windows)
    assert np.array_equal(gy, start.y)
    assert np.array_equal(gf, of), (gf, of)
    assert np.array_equal(ga, last.active)
    assert np.array_equal(gx, last.x), np.max(np.abs(gx - last.x))
    assert np.array_equal(gt, last.t), np.max(np.abs(gt - last.t))
    a, b = chain_order(olog), chain_order(glog)
    assert len(a) == len(b)
    for f in ("leg", "c", "i", "j", "t", "tau", "xi", "xj"):
        assert np.array_equal(a[f], b[f]), f
    assert st["liftings"] == len(olog)
    # per-window flags (windows whose isolated claim sets met), counted
    assert st["conflict_windows"] == last.window_flags
    assert st["horizon_asserts"] == 0
    assert st["order_errors"] == 0
    return gf, st


@pytest.mark.parametrize("seed", range(10))
def test_config1_lattice_n256(seed):
    """N=256 (16x16 lattice, jitter 0.01), eta=0.70, 4 chains, ell=0.5, 8 legs."""
    s = synth.lattice_start(16, 0.70, 4, seed=seed)
    assert_parity(s, 0.5, 8)


def test_config2_lattice_n16384_few_legs():
    """N=16384 (128x128), eta=0.708, 128 chains, ell=1: the first legs in full."""
    s = synth.lattice_start(128, 0.708, 128, seed=7)
    flags, st = assert_parity(s, 1.0, 3)
    assert st["liftings"] > 5000


def test_config3_lattice_n1m_one_leg():
    """N=2^20 (1024x1024), eta=0.72, 1024 chains, ell=1: one full leg."""
    s = synth.lattice_start(1024, 0.72, 1024, seed=3)
    assert_parity(s, 1.0, 1)


@pytest.mark.parametrize("seed,k", [(1, 1), (2, 3), (3, 8)])
def test_random_2d_starts(seed, k):
    """Non-lattice starts: cross-row liftings through the j+/j- corridors."""
    s = synth.rsa_start(300, 0.45, k, seed=seed)
    assert_parity(s, 2.0, 4)


def test_conflict_free_legs_take_the_parallel_path():
    """Sparse chains on a big lattice: most legs have no conflict and then the
    result comes straight from the parallel pass."""
    s = synth.lattice_start(96, 0.70, 2, seed=11)
    flags, _ = assert_parity(s, 0.3, 6)
    assert flags.sum() < len(flags)


def test_cells_per_side_does_not_change_positions():
    """The cell size changes the flags (claims) but not the physics."""
    s = synth.lattice_start(24, 0.70, 6, seed=5)
    f1, st1 = assert_parity(s, 0.5, 3, nc=O.default_cells(s.box))
    f2, st2 = assert_parity(s, 0.5, 3, nc=16)  # a/d = 1.55: 8 slots per cell


def test_edge_small_box_three_cells():
    """Smallest box: three cells per side, chains wrapping around."""
    s = synth.rsa_start(5, 0.35, 2, seed=4)
    assert O.default_cells(s.box) == 3
    assert_parity(s, 1.5, 4)


def test_edge_every_disk_active():
    """k = N: no static disk is left, every chain stalls at once."""
    s = synth.lattice_start(4, 0.6, 16, seed=2)
    gf, st = assert_parity(s, 0.7, 2)
    assert st["liftings"] == 0


def test_edge_single_chain_long_leg():
    """One chain with ell larger than the box side."""
    s = synth.lattice_start(6, 0.5, 1, seed=9)
    assert s.box < 10
    assert_parity(s, 12.0, 2)


def test_errors_are_reported():
    s = synth.lattice_start(8, 0.6, 2, seed=1)
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.System(s.x, s.y, [0, 0], s.box, 1.0)
    assert e.value.code == ecmc.ECMC_EINVAL
    bad = s.x.copy()
    bad[3] = s.box
    with pytest.raises(ecmc.EcmcError):
        ecmc.System(bad, s.y, [0, 1], s.box, 1.0)
    # undo records too small for the leg: a clean ECAPACITY, not a fault
    sysm = ecmc.System(s.x, s.y, [0, 1], s.box, 5.0, undo_cap=2)
    with pytest.raises(ecmc.EcmcError) as e:
        sysm.run(1)
    assert e.value.code == ecmc.ECMC_ECAPACITY
    sysm.close()


@pytest.mark.parametrize("m,k,ell,seed", [(32, 64, 1.0, 1), (32, 200, 1.0, 2), (48, 48, 3.0, 3)])
def test_dense_chains_merge_components(m, k, ell, seed):
    """Many chains per disk: conflict components with many members that meet
    other chains while being redone, so repair needs several rounds."""
    s = synth.lattice_start(m, 0.70, k, seed=seed)
    flags, st = assert_parity(s, ell, 3)
    assert flags.all()
    assert st["repaired_chains"] > k


@pytest.mark.parametrize("seed", [21, 22])
def test_dense_random_2d_components(seed):
    s = synth.rsa_start(400, 0.5, 40, seed=seed)
    flags, st = assert_parity(s, 1.5, 3)
    assert flags.all()


@pytest.mark.parametrize("windows", [2, 5, 16])
@pytest.mark.parametrize("seed", [0, 3])
def test_claim_windows_config1(windows, seed):
    """Claim windows: same liftings and positions as one window, flags equal to
    the oracle's windowed flags."""
    s = synth.lattice_start(16, 0.70, 4, seed=seed)
    assert_parity(s, 0.5, 8, windows=windows)


@pytest.mark.parametrize("windows", [4, 32])
def test_claim_windows_dense_components(windows):
    s = synth.lattice_start(32, 0.70, 200, seed=2)
    assert_parity(s, 1.0, 3, windows=windows)


def test_claim_windows_config2_and_random():
    s = synth.lattice_start(128, 0.708, 128, seed=7)
    assert_parity(s, 1.0, 2, windows=8)
    r = synth.rsa_start(400, 0.5, 40, seed=21)
    assert_parity(r, 1.5, 3, windows=6)


def test_claim_windows_config3_one_leg():
    s = synth.lattice_start(1024, 0.72, 4096, seed=3)
    assert_parity(s, 1.0, 1, windows=16)


def test_repairs_by_continuation_and_takeover_n1m():
    """N = 2^20 with 16384 chains: most conflict components are finished by
    continuing their blocked chains (and taking over chains in no component);
    the rest by rollback and replay. Bit-exact either way."""
    s = synth.lattice_start(1024, 0.72, 16384, seed=5)
    flags, st = assert_parity(s, 1.0, 1, windows=4)
    assert flags.all()
    assert 0 < st["continued_chains"] < st["repaired_chains"]


def test_repairs_by_continuation_random_2d():
    """Cross-row liftings: continuation fails where chains really interact."""
    s = synth.rsa_start(3000, 0.45, 120, seed=13)
    flags, st = assert_parity(s, 1.5, 3, windows=3)
    assert st["repaired_chains"] > 0


@pytest.mark.parametrize("kind", ["lattice", "rsa"])
def test_direction_alternation_equals_oracle_on_swapped_frame(kind):
    """Legs alternating +x / +y: a +y leg is the oracle's +x leg with x and y
    exchanged. Positions and active disks bit for bit after every leg."""
    if kind == "lattice":
        s = synth.lattice_start(24, 0.70, 12, seed=4)
        ell = 1.0
    else:
        s = synth.rsa_start(500, 0.45, 20, seed=6)
        ell = 1.5
    sysm = ecmc.System(s.x, s.y, s.active, s.box, ell)
    x, y, act = s.x.copy(), s.y.copy(), s.active.copy()
    for leg in range(6):
        d = leg % 2
        sysm.set_direction(d)
        sysm.run(1)
        if d == 0:
            r = O.run_leg(x, y, act, s.box, ell, log=False)
            x, act = r.x, r.active
        else:
            r = O.run_leg(y, x, act, s.box, ell, log=False)
            y, act = r.x, r.active
        gx, gy, _, ga = sysm.positions()
        assert np.array_equal(gx, x) and np.array_equal(gy, y), leg
        assert np.array_equal(ga, act), leg
    st = sysm.stats()
    assert st["horizon_asserts"] == 0 and st["order_errors"] == 0
    sysm.close()


@pytest.mark.parametrize("seed,windows", [(1, 1), (2, 1), (3, 2), (4, 3)])
def test_staggered_rows_skip_and_cross(seed, windows):
    """Rows in close pairs, the pairs far apart in y: a scan skips the row on
    the far side of its pair (claimed weakly: the flag still sees it), and
    chains lift between the two rows of a pair, taking over weak claims,
    their own and other chains'."""
    s = synth.staggered_start(16, 0.5, 12, seed, row_shift=0.05, pair_shift=0.15)
    assert_parity(s, 1.5, 6, windows=windows)


def test_staggered_rows_dense_chains():
    s = synth.staggered_start(24, 0.5, 96, 7, row_shift=0.05, pair_shift=0.15)
    flags, st = assert_parity(s, 1.0, 4)
    assert st["repaired_chains"] > 0


@pytest.mark.parametrize("seed", [8, 9])
def test_staggered_rows_random_shifts(seed):
    """Rows moved by independent shifts: some neighbours within d in y, some not."""
    s = synth.staggered_start(32, 0.5, 24, seed, row_shift=0.2)
    assert_parity(s, 1.5, 4)


def test_staggered_rows_direction_alternation():
    """The skipped rows are recomputed for the transposed frame; flags, positions
    and active disks equal the oracle's on the exchanged coordinates."""
    s = synth.staggered_start(16, 0.5, 10, 5, row_shift=0.05, pair_shift=0.15)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.2)
    x, y, act = s.x.copy(), s.y.copy(), s.active.copy()
    for leg in range(6):
        d = leg % 2
        sysm.set_direction(d)
        f, _ = sysm.run(1)
        if d == 0:
            r = O.run_leg(x, y, act, s.box, 1.2, log=False)
            x, act = r.x, r.active
        else:
            r = O.run_leg(y, x, act, s.box, 1.2, log=False)
            y, act = r.x, r.active
        gx, gy, _, ga = sysm.positions()
        assert np.array_equal(gx, x) and np.array_equal(gy, y), leg
        assert np.array_equal(ga, act), leg
        assert int(f[0]) == r.flag, leg
    sysm.close()
