"""The two FP32 shortcuts of the CUDA path, checked numerically on the CPU.

1. The spot-diagram reduction bins r^2 in FP32 (dx = x - fl(cx), r2 =
   fma(dx, dx, fl(dy * dy)), f = fl(r2 * fl(scale))) and trusts the bin only
   where its error bound delta (computed per window from the centroid and the
   range) is below 1/2.  Here every photon's |f_FP32 - f_exact| must stay
   below delta, on spots placed to stress the bound.
2. The device photon source screens each hexagon candidate in FP32 and
   decides in FP64 only within 1e-5 a of the boundary; the FP32 hexagon
   measure must stay within 2e-6 a of the FP64 one.

numpy float32 arithmetic rounds once per operation, as the device does; the
fused multiply-add is emulated exactly (the product of two floats is exact in
FP64, then one rounding to FP32).
"""
import math

import numpy as np

F = np.float32
K_BINS = 4096


def fmaf(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def delta_bound(cx, cy, scale):
    """The bound of the reduction's finish step, restated from its derivation."""
    u = 2.0 ** -24
    R2 = (K_BINS + 2) / scale
    R = math.sqrt(R2)
    ex = u * abs(cx) * (1 + u) + u * R
    ey = u * abs(cy) * (1 + u) + u * R
    E = R + ex + ey
    err = ex * (2 * R + ex) + ey * (2 * R + ey) + (2 * u + u * u) * E * E
    return scale * err + (2 * u + u * u) * scale * (R2 + err)


def test_fp32_binning_error_stays_below_the_bound():
    rng = np.random.default_rng(5)
    cases = [((0.3, -1.02), 0.02), ((0.0, 0.0), 0.03), ((-1.5, 2.0), 0.005), ((1.0, 1.0), 1e-4), ((12.0, -7.0), 0.05)]
    for (mx, my), sig in cases:
        x = (rng.normal(mx, sig, 400_000)).astype(F)
        y = (rng.normal(my, sig, 400_000)).astype(F)
        xd, yd = x.astype(np.float64), y.astype(np.float64)
        cx, cy = xd.mean(), yd.mean()
        ms = ((xd - cx) ** 2 + (yd - cy) ** 2).mean()
        scale = K_BINS / (64.0 * ms)
        delta = delta_bound(cx, cy, scale)
        dx = (x - F(cx)).astype(F)
        dy = (y - F(cy)).astype(F)
        r2f = fmaf(dx, dx, (dy * dy).astype(F))
        ff = (r2f * F(scale)).astype(F).astype(np.float64)
        fe = ((xd - cx) ** 2 + (yd - cy) ** 2) * scale  # exact to FP64 rounding
        inside = fe < K_BINS + 2
        err = np.max(np.abs(ff[inside] - fe[inside]))
        assert err <= delta, ((mx, my), sig, err, delta)
        if delta < 0.1:  # the bound is not vacuous where the fast path is used
            assert err > 0.0


def test_fp32_hexagon_screen_stays_within_its_band():
    rng = np.random.default_rng(9)
    n = 2_000_000
    for a in (0.025, 1.0, 12.0):
        R = a * 2.0 / math.sqrt(3.0)
        w0 = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
        w1 = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
        # FP64 definition
        u0 = (w0.astype(np.float64) + 0.5) * 2.0 ** -32
        u1 = (w1.astype(np.float64) + 0.5) * 2.0 ** -32
        x = (2.0 * u0 - 1.0) * a
        y = (2.0 * u1 - 1.0) * R
        s60 = 0.86602540378443864676
        m64 = np.maximum(np.abs(x), np.maximum(np.abs(0.5 * x + s60 * y), np.abs(-0.5 * x + s60 * y)))
        # FP32 screen, one rounding per operation (fused forms are at least as accurate)
        u0f = ((w0.astype(F) + F(0.5)) * F(2.0 ** -32)).astype(F)
        u1f = ((w1.astype(F) + F(0.5)) * F(2.0 ** -32)).astype(F)
        xf = ((F(2.0) * u0f - F(1.0)) * F(a)).astype(F)
        yf = ((F(2.0) * u1f - F(1.0)) * F(R)).astype(F)
        hx, sy = (F(0.5) * xf).astype(F), (F(s60) * yf).astype(F)
        mf = np.maximum(np.abs(xf), np.maximum(np.abs(hx + sy), np.abs(sy - hx))).astype(np.float64)
        assert np.max(np.abs(mf - m64)) <= 2e-6 * a, a
        # the screen never decides against the FP64 test outside its band
        a32 = float(F(a))
        sure_in = mf < a32 * float(F(1.0) - F(1e-5))
        sure_out = mf > a32 * float(F(1.0) + F(1e-5))
        assert np.all(m64[sure_in] <= a) and np.all(m64[sure_out] > a)
