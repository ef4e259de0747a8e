"""The cell scan's stop rule on its FP32 image (host-side check of the bound).

The scan asks, for each next column m, whether thr(m) = ((m a) - fx) - d lies
above lim = RN(cur + eps) (all FP64). It first evaluates the same expression in
FP32: thr_f = ((m af - fxf) - df), lim_f = trunc32(cur) + epsf, with af, df,
epsf the FP32 roundings and fxf = fx truncated toward zero. It trusts the FP32
answer only when thr_f - lim_f lies farther than stop_e = 2^-20 (L + a + d +
ell + eps + 1) from 0, which is 4x the worst-case error of the image. This
emulates that sequence of IEEE operations in numpy (float32 arithmetic rounds
to nearest like the device's __f*_rn intrinsics) and checks the bound and the
decisions against the FP64 rule over the box sizes the configurations use.
"""
import math

import numpy as np
import pytest

f32 = np.float32


def trunc32(v):
    """v rounded toward zero to float32 (the device's integer-pipe conversion)."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    over = np.abs(f.astype(np.float64)) > np.abs(v)
    f = np.where(over, np.nextafter(f, np.float32(0)), f)
    return f.astype(np.float32)


def image(m, fx, cur, a, d, eps):
    af, df, epsf = f32(a), f32(d), f32(eps)
    thr_f = (f32(m).astype(f32) * af - trunc32(fx)) - df
    lim_f = trunc32(cur) + epsf
    return (thr_f - lim_f).astype(np.float64)


def exact(m, fx, cur, a, d, eps):
    thr = ((m.astype(np.float64) * a) - fx) - d
    lim = cur + eps
    return thr, lim


@pytest.mark.parametrize("n,eta,ell", [(256, 0.70, 0.5), (16384, 0.708, 1.0),
                                       (1 << 20, 0.72, 1.0), (1 << 22, 0.62, 1.0),
                                       (1024, 0.60, 3.0)])
def test_fp32_stop_image_is_exact_outside_its_band(n, eta, ell):
    d = 1.0
    L = math.sqrt(n * math.pi * d * d / (4 * eta))
    nc = int(L / (d * (1.0 + 2.0 ** -20)))
    a = L / nc
    eps = math.ldexp(L, -30)
    stop_e = float(f32(math.ldexp(L + a + d + ell + eps + 1.0, -20)))
    rng = np.random.default_rng(n)
    k = 400_000
    m = np.concatenate([rng.integers(0, 4, k // 2), rng.integers(0, nc, k // 2)])
    fx = rng.random(k) * a
    fx[: k // 8] = -rng.random(k // 8) * 1e-13  # a disk a rounding step left of its column
    cur = rng.random(k) * ell
    cur[k // 8: k // 4] = ell
    diff_f = image(m, fx, cur, a, d, eps)
    thr, lim = exact(m, fx, cur, a, d, eps)
    # the error of the image stays below a quarter of the band
    assert np.max(np.abs(diff_f - (thr - lim))) < stop_e / 4
    # and outside the band its decision is the FP64 one (thr >= 0 and thr > lim)
    beyond = (thr >= 0) & (thr > lim)
    assert np.all(beyond[diff_f > stop_e])
    assert not np.any(beyond[diff_f < -stop_e])
    # "scanned in any case" (thr <= eps) is claimed only where certain
    thr_f = (f32(m).astype(f32) * f32(a) - trunc32(fx)) - f32(d)
    sure = thr_f < (f32(eps) - f32(stop_e))
    assert np.all(thr[sure] <= eps)
    # near the decision the band does send cases to the FP64 path
    near = np.abs(thr - lim) < stop_e
    if near.any():
        assert np.all(np.abs(diff_f[near]) <= 2 * stop_e)
