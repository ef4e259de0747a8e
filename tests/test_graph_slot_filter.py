"""The constraint-graph build's FP32 slot filter, checked on the host.

While it scans the cells ahead of disk i, the build skips a slot j without any
FP64 work when the FP32 image of the minimum-image |dy| -- y_i and y_j rounded
to FP32, |RN32(y_j - y_i)|, and L - that where smaller -- exceeds
dcut = RN32(d (1 + 10^-3) + 10^-6 L): a margin far above the image's error
(a few 2^-24 L). The exact test is the FP64 minimum image |dy| < d (the
corridors). This emulates both in numpy and checks that a skipped slot is never
in a corridor, that the filter skips nearly every slot beyond 1.01 d, and that
without the L-proportional part of the margin the filter would be unsafe on
large boxes where d is not on the FP32 grid of y (so the check can fail)."""
import math

import numpy as np
import pytest

f32 = np.float32


def image_skips(yi, yj, L, dcut):
    ayf0 = np.abs((f32(yj) - f32(yi)).astype(f32)).astype(f32)
    ayf = np.minimum(ayf0, (f32(L) - ayf0).astype(f32))
    return ayf > f32(dcut)


def exact_ay(yi, yj, L):
    ay = np.abs(yj - yi)  # RN(y_j - y_i), then |.|
    la = L - ay
    return np.where(la < ay, la, ay)


@pytest.mark.parametrize("d", [1.0, 0.7, 1.3])
@pytest.mark.parametrize("n_disks,eta", [(16384, 0.708), (1 << 20, 0.72), (4 << 20, 0.70)])
def test_skipped_slots_are_in_no_corridor(n_disks, eta, d):
    L = math.sqrt(n_disks * math.pi * d * d / (4.0 * eta))
    dcut = float(f32(d * (1.0 + 1e-3) + L * 1e-6))
    rng = np.random.default_rng(n_disks)
    n = 600_000
    yi = rng.uniform(0.0, L, n)
    # |dy| around d (either sign, across the periodic edge too) and generic
    off = np.concatenate([d + rng.uniform(-2e-3, 2e-3, n // 2), rng.uniform(0.0, 4 * d, n - n // 2)])
    sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    yj = np.mod(yi + sign * off, L)
    skip = image_skips(yi, yj, L, dcut)
    ay = exact_ay(yi, yj, L)
    wrong = skip & (ay < d)
    assert not wrong.any(), (yi[wrong][:3], yj[wrong][:3])
    # the filter does its job: slots clearly out of the corridors are skipped
    far = ay > 1.01 * d
    assert far.sum() > 100_000 and skip[far].all()
    if n_disks >= (1 << 20) and d != 1.0:
        # a margin of 10^-6 d alone would not cover the FP32 error at this box
        # size near |dy| = d (with d = 1 the FP32 grid of y meets d exactly,
        # and the image near d is exact)
        tight = image_skips(yi, yj, L, float(f32(d * (1.0 + 1e-6)))) & (ay < d)
        assert tight.any()
