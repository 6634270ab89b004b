"""The FP32 screen of the element-pair test (CPU, numpy float32): boxes rounded outwards to
FP32, the screened distance compared against reach -/+ margin with
margin = 8 * 2^-23 * (max |coordinate| + reach), must never decide differently from the FP64
test of eq. (mindist); inside the window the FP64 test decides.  This checks the margin
argument on adversarial boxes whose FP64 distance sits within a few ulps of the threshold,
on domains far from the origin where the FP32 rounding is largest."""
import numpy as np
import pytest

F32_EPS = 1.1920928955078125e-07  # 2^-23


def _down(x):
    f = x.astype(np.float32)
    up = f.astype(np.float64) > x
    f[up] = np.nextafter(f[up], np.float32(-np.inf))
    return f


def _up(x):
    f = x.astype(np.float32)
    dn = f.astype(np.float64) < x
    f[dn] = np.nextafter(f[dn], np.float32(np.inf))
    return f


def _mindist64(lo1, hi1, lo2, hi2):
    d = np.maximum(lo1 - hi2, lo2 - hi1)
    return np.maximum(d.max(axis=-1), 0.0)


def _screen(lo1, hi1, lo2, hi2, reach, cmax):
    margin = 8.0 * F32_EPS * (cmax + reach)
    lo_t, hi_t = np.float32(reach - margin), np.float32(reach + margin)
    f1l, f1h, f2l, f2h = _down(lo1), _up(hi1), _down(lo2), _up(hi2)
    d = np.maximum(f1l - f2h, f2l - f1h)  # float32 arithmetic
    mf = np.maximum(d.max(axis=-1), np.float32(0))
    return np.where(mf < lo_t, 1, np.where(mf > hi_t, 0, -1))  # -1: FP64 decides


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("origin", [0.0, 1.0, 1000.0, -3.0e5])
def test_screen_never_contradicts_the_fp64_test(dim, origin):
    rng = np.random.default_rng(11 + dim)
    n = 200_000
    reach = 0.05
    size = rng.uniform(1e-3, 2e-2, (n, dim))
    lo2 = origin + rng.uniform(0, 1, (n, dim))
    hi2 = lo2 + size
    # place box 1 so that its FP64 distance along a random axis is reach + t, t within a few
    # ulps of the threshold (and a spread of wider offsets)
    ax = rng.integers(0, dim, n)
    t = np.where(rng.random(n) < 0.5, rng.integers(-64, 65, n) * np.spacing(reach + abs(origin) + 1),
                 rng.uniform(-2 * reach, 2 * reach, n))
    lo1 = lo2 + rng.uniform(-0.5, 0.5, (n, dim)) * size
    hi1 = lo1 + rng.uniform(1e-3, 2e-2, (n, dim))
    idx = np.arange(n)
    w1 = hi1[idx, ax] - lo1[idx, ax]
    lo1[idx, ax] = hi2[idx, ax] + reach + t
    hi1[idx, ax] = lo1[idx, ax] + w1
    cmax = float(np.abs(np.concatenate([lo1, hi1, lo2, hi2])).max())
    exact = _mindist64(lo1, hi1, lo2, hi2) < reach
    scr = _screen(lo1, hi1, lo2, hi2, reach, cmax)
    decided = scr >= 0
    assert np.all(scr[decided] == exact[decided])
    margin = 8 * F32_EPS * (cmax + reach)
    if margin < 0.1 * reach:
        # the window is narrow: every pair clear of it is decided in FP32
        far = np.abs(_mindist64(lo1, hi1, lo2, hi2) - reach) > 2 * margin
        assert far.any() and decided[far].all()
        assert decided.mean() > 0.4
    # (far from the origin FP32 cannot resolve the reach: the window covers everything and
    # the FP64 test decides every pair, which is still exact)
