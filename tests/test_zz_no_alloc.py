"""The leg entry point that allocates nothing (ecmc_leg_noalloc).

It serves callers that cannot allocate device memory -- code inside a
framework whose caching allocator owns the device heap, real-time loops, and
plug-ins that only receive pointers. It must give, bit for bit, what the
allocating entry points give for the same leg. Collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2004_11040_gb300 import ecmc, synth

pytestmark = pytest.mark.gpu


def _compare_two_legs(start, ell, cells_per_side=0):
    torch = pytest.importorskip("torch")
    stream = torch.cuda.current_stream()
    ref = ecmc.System(start.x, start.y, start.active, start.box, ell,
                      cells_per_side=cells_per_side, stream=stream)
    x = torch.tensor(start.x, dtype=torch.float64, device="cuda")
    y = torch.tensor(start.y, dtype=torch.float64, device="cuda")
    act = torch.tensor(start.active, dtype=torch.int32, device="cuda")
    t = torch.empty_like(x)
    flags = []
    for call in range(2):  # two calls in a row, the second continuing the first
        before = ref.stats()["liftings"]
        rflags, _ = ref.run(1)
        rx, _, rt, ra = ref.positions()
        flag, lifts = ecmc.ecmc_leg_noalloc(start.n, start.box, start.d, ell, start.k,
                                            cells_per_side, x, y, act, t, stream)
        assert np.array_equal(x.cpu().numpy(), rx), call
        assert np.array_equal(t.cpu().numpy(), rt), call
        assert np.array_equal(act.cpu().numpy(), ra), call
        assert flag == int(rflags[0]), call
        assert lifts == ref.stats()["liftings"] - before, call
        flags.append(flag)
    ref.close()
    return flags


def test_noalloc_leg_equals_allocating_path_with_conflicts():
    s = synth.lattice_start(32, 0.70, 12, seed=4)
    flags = _compare_two_legs(s, 0.8)
    assert any(flags)  # the repair path ran inside the no-allocation call


def test_noalloc_leg_equals_allocating_path_sparse():
    s = synth.lattice_start(64, 0.72, 2, seed=8)
    _compare_two_legs(s, 0.5)


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    n = 4_000_000  # needs far more than the fixed scratch array
    box = synth.box_side(n, 0.7)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    ids = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.ecmc_leg_noalloc(n, box, 1.0, 1.0, 2, 0, dummy, dummy, ids)
    assert e.value.code == ecmc.ECMC_EINVAL
