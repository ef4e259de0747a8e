"""Contexts built on blocks from the device memory cache: the blocks a
destroyed context gives back hold its state, and a context that takes them
must still give the oracle's result bit for bit (nothing may rely on fresh
device memory). Also the cache's books through the C ABI."""
import numpy as np
import pytest

from paper_2004_11040_gb300 import ecmc, synth

from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu

DEFAULT_LIMIT = 4 << 30


def _dirty_the_cache(start_like, legs, graph=False, windows=1, log=True):
    """Runs another system of the same sizes (other seed, so other cells,
    records, claims and repairs), then destroys it: its blocks are cached.
    Returns the device bytes it held (the log capacity is the parity
    helper's, so the next context asks for blocks of the same sizes)."""
    other = synth.lattice_start(start_like.m, start_like.eta, start_like.k,
                                seed=start_like.seed + 101)
    sysm = ecmc.System(other.x, other.y, other.active, other.box, 1.0, d=other.d, log=log,
                       log_cap=max(1 << 16, 64 * other.k * legs * 64), graph=graph,
                       windows=windows)
    flags, done = sysm.run(legs)
    assert done == legs and flags.any()  # it had conflicts (repairs wrote scratch)
    sysm.positions()
    held = sysm.stats()["device_bytes"]
    sysm.close()
    return held


class _Start:
    def __init__(self, m, eta, k, seed):
        self.m, self.eta, self.k, self.seed = m, eta, k, seed
        self.s = synth.lattice_start(m, eta, k, seed=seed)


@pytest.mark.parametrize("windows", [1, 4])
def test_reused_blocks_give_the_oracle_result(windows):
    ecmc.ecmc_set_cache_limit(DEFAULT_LIMIT)
    st = _Start(64, 0.70, 64, 3)
    held = _dirty_the_cache(st, 3, windows=windows)
    before = ecmc.ecmc_cache_info()
    assert before["cached_bytes"] >= held
    _, stats = assert_parity(st.s, 1.0, 3, windows=windows)
    # the same sizes: the context was built on the dirty context's blocks
    assert stats["device_bytes"] == held
    after = ecmc.ecmc_cache_info()
    assert after["misses"] == before["misses"]
    assert after["hits"] > before["hits"]


def test_reused_blocks_graph_mode():
    ecmc.ecmc_set_cache_limit(DEFAULT_LIMIT)
    st = _Start(64, 0.70, 64, 5)
    held = _dirty_the_cache(st, 3, graph=True, log=False)
    h0 = ecmc.ecmc_cache_info()["hits"]
    s = st.s
    g = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d, graph=True)
    fg, _ = g.run(3)
    xg, _, tg, ag = g.positions()
    assert g.stats()["device_bytes"] == held
    g.close()
    assert ecmc.ecmc_cache_info()["hits"] > h0
    ref = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d)  # the cell scan
    fr, _ = ref.run(3)
    xr, _, tr, ar = ref.positions()
    ref.close()
    assert np.array_equal(fr, fg)
    assert np.array_equal(xr, xg) and np.array_equal(tr, tg) and np.array_equal(ar, ag)


def test_cache_books_and_limit():
    ecmc.ecmc_set_cache_limit(DEFAULT_LIMIT)
    s = synth.lattice_start(32, 0.70, 16, seed=0)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d)
    sysm.run(1)
    sysm.positions()
    held = sysm.stats()["device_bytes"]
    info = ecmc.ecmc_cache_info()
    assert info["in_use_bytes"] >= held
    sysm.close()
    info2 = ecmc.ecmc_cache_info()
    assert info2["in_use_bytes"] <= info["in_use_bytes"] - held
    assert info2["cached_bytes"] >= held
    # the same sizes again: no new device allocation
    m0 = info2["misses"]
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d)
    sysm.run(1)
    sysm.positions()
    sysm.close()
    assert ecmc.ecmc_cache_info()["misses"] == m0
    # limit 0: nothing is kept
    ecmc.ecmc_set_cache_limit(0)
    assert ecmc.ecmc_cache_info()["cached_bytes"] == 0
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d)
    sysm.run(1)
    sysm.close()
    assert ecmc.ecmc_cache_info()["cached_bytes"] == 0
    with pytest.raises(ecmc.EcmcError):
        ecmc.ecmc_set_cache_limit(-1)
    ecmc.ecmc_set_cache_limit(DEFAULT_LIMIT)
