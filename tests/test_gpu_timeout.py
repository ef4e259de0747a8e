"""The bounded device waits (ECMC_ETIMEOUT): a wait limit far below the
time one leg takes makes the persistent kernel give up at a grid barrier;
the call returns ECMC_ETIMEOUT instead of hanging, and the context can be
destroyed. Every wait of the launch is bounded, so nothing can hang."""
import numpy as np
import pytest

from paper_2004_11040_gb300 import ecmc, synth

pytestmark = pytest.mark.gpu


def test_short_wait_limit_returns_timeout_and_context_is_destroyed():
    s = synth.lattice_start(256, 0.72, 2048, seed=1)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0)
    sysm.set_wait_limit(1)  # 1 ns: any block that waits at all gives up
    with pytest.raises(ecmc.EcmcError) as e:
        sysm.run(5)
    assert e.value.code == ecmc.ECMC_ETIMEOUT
    sysm.close()
    # the device is usable afterwards
    t = synth.lattice_start(16, 0.70, 4, seed=0)
    other = ecmc.System(t.x, t.y, t.active, t.box, 0.5)
    flags, done = other.run(2)
    assert done == 2
    other.close()


def test_wait_limit_rejects_out_of_range():
    s = synth.lattice_start(16, 0.70, 4, seed=0)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 0.5)
    for bad in (0, 61 * 10**9):
        with pytest.raises(ecmc.EcmcError) as e:
            sysm.set_wait_limit(bad)
        assert e.value.code == ecmc.ECMC_EINVAL
    sysm.close()
