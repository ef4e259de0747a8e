"""The row continuation's FP32 image of the horizon condition (Eq. 2), checked
on the host.

For a scanned disk j (not the target) with t_j != 0 the continuation needs
Eq. 2's lower bound: sb = RN(RN(x_j - x_k) - d) >= 0 and RN(t + sb) > t_j, with
x_k and t the active disk's position and the chain's time. It first evaluates
the same expression in FP32 -- x_j, x_k, t and t_j truncated to FP32, d rounded
-- and trusts the answer "holds" when both the image of sb and the image of
t + sb - t_j exceed stop_e = 2^-20 (L + a + d + ell + eps + 1) (the band of the
stop rule's image); anything else is decided in FP64. Each of the image's six
roundings errs by at most 2^-23 of a term below L + d + ell, so the image is
within about 2^-21 (L + d + ell) of the exact value: "holds" on the image
implies "holds" exactly. This emulates the device's operation sequence in
numpy (float32 arithmetic rounds to nearest like __fadd_rn / __fsub_rn) and
checks the implication on generic and near-boundary cases, and that a band
64 times narrower would not be safe (so the check can fail)."""
import math

import numpy as np
import pytest

from test_stop_image import trunc32

f32 = np.float32


def image_holds(xk, xj, t, tj, d, stop_e):
    pxf, xkf, df = trunc32(xj), trunc32(xk), f32(d)
    sbf = ((pxf - xkf).astype(f32) - df).astype(f32)
    mf = ((trunc32(t) + sbf).astype(f32) - trunc32(tj)).astype(f32)
    return (sbf > f32(stop_e)) & (mf > f32(stop_e))


def exact_holds(xk, xj, t, tj, d):
    sb = (xj - xk) - d  # float64, round to nearest: the device's __dsub_rn
    return (sb >= 0.0) & ((t + sb) > tj)


def cases(rng, L, d, ell, n):
    """Generic and near-boundary (x_k, x_j, t, t_j): x_j ahead of x_k by d plus a
    gap of up to a few d, times in [0, ell), t_j at, above and below t + gap."""
    xk = rng.uniform(0.0, L - 4 * d, n)
    gap = np.concatenate([rng.uniform(0.0, 3 * d, n // 2),
                          rng.uniform(0.0, 1e-4, n - n // 2)])  # near sb = 0
    xj = xk + d + gap
    t = rng.uniform(0.0, ell, n)
    scale = np.concatenate([np.full(n // 3, 1.0), np.full(n // 3, 1e-4),
                            np.full(n - 2 * (n // 3), 1e-6)])
    tj = t + gap + scale * rng.uniform(-1.0, 1.0, n)  # around Eq. 2's boundary
    keep = (tj > 0.0) & (tj < ell) & (xj < L)
    return xk[keep], xj[keep], t[keep], tj[keep]


@pytest.mark.parametrize("n_disks,eta", [(16384, 0.708), (1 << 20, 0.72), (4 << 20, 0.70)])
def test_image_holds_implies_exact(n_disks, eta):
    d, ell = 1.0, 1.0
    L = math.sqrt(n_disks * math.pi * d * d / (4.0 * eta))
    a = L / round(math.sqrt(n_disks))
    eps = math.ldexp(L, -30)
    stop_e = float(f32(math.ldexp(L + a + d + ell + eps + 1.0, -20)))
    rng = np.random.default_rng(n_disks)
    xk, xj, t, tj = cases(rng, L, d, ell, 400_000)
    img = image_holds(xk, xj, t, tj, d, stop_e)
    ex = exact_holds(xk, xj, t, tj, d)
    bad = img & ~ex
    assert not bad.any(), (xk[bad][:3], xj[bad][:3], t[bad][:3], tj[bad][:3])
    # and it decides every case that holds with a margin of a few bands (the
    # FP64 fallback is for the cases near the boundary only)
    sb = (xj - xk) - d
    clear = (sb > 4 * stop_e) & ((t + sb) - tj > 4 * stop_e)
    assert clear.sum() > 10_000 and img[clear].all()
    # and a band 64 times narrower than stop_e would let wrong answers through
    narrow = image_holds(xk, xj, t, tj, d, stop_e / 64) & ~ex
    assert narrow.any()
