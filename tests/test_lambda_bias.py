"""Lambda-side potentials (double well, pH potential, partition function correction): the
oracle against closed forms, and the library's host-side correction against the oracle."""
import ctypes
import math

import numpy as np
import pytest

from oracle import lambda_bias as lb


def test_spline_values_and_slopes_at_the_knots():
    a0, a1, h, d, kw = 0.0, 1.0, 7.5, -2.25, 900.0
    for l, v in ((a0, 0.0), (0.5, h), (a1, d)):
        V, dV = lb.potential(l, a0, a1, h, d, kw)
        assert V == pytest.approx(v, abs=1e-14) and dV == pytest.approx(0.0, abs=1e-12)
    # continuity across the knots and the walls, and the walls' slopes
    for l in (a0, 0.5, a1):
        for e in (1e-9,):
            assert lb.potential(l - e, a0, a1, h, d, kw)[0] == pytest.approx(lb.potential(l + e, a0, a1, h, d, kw)[0],
                                                                              abs=1e-6)
    assert lb.potential(-0.1, a0, a1, h, d, kw)[1] == pytest.approx(-90.0)
    assert lb.potential(1.1, a0, a1, h, d, kw)[0] == pytest.approx(d + 0.5 * 900.0 * 0.01)
    # derivative by central differences inside the pieces
    for l in (0.13, 0.37, 0.61, 0.94, -0.05, 1.07):
        fd = (lb.potential(l + 1e-7, a0, a1, h, d, kw)[0] - lb.potential(l - 1e-7, a0, a1, h, d, kw)[0]) / 2e-7
        assert fd == pytest.approx(lb.potential(l, a0, a1, h, d, kw)[1], rel=1e-6, abs=1e-6)


def test_pfc_symmetric_case_is_zero():
    assert lb.pfc_delta(pH=4.0, pKa=4.0, h=8.0, kT=2.494339) == pytest.approx(0.0, abs=1e-9)


def _trapezoid_log10_ratio(a, b, c, h, d, kT, npts=240001):
    """log10(Z_deprot / Z_prot) by a plain trapezoid rule on a uniform grid over [a, c]
    split at b (the grid puts a node on b)."""
    l = np.linspace(a, c, npts)
    V = np.array([lb.potential(x, 0.0, 1.0, h, d, 1000.0)[0] for x in l])
    w = np.exp(-V / kT)
    mid = int(round((b - a) / (c - a) * (npts - 1)))
    assert abs(l[mid] - b) < 1e-12
    zp = np.trapezoid(w[: mid + 1], l[: mid + 1])
    zd = np.trapezoid(w[mid:], l[mid:])
    return math.log10(zd / zp)


@pytest.mark.parametrize("dpH", [-1.5, -0.3, 0.7, 2.0])
def test_pfc_reaches_the_henderson_hasselbalch_ratio(dpH):
    """Independent check of Sec. 2.3's condition: with the corrected offset, the partition
    functions over [0, 0.5] and [0.5, 1], by a plain trapezoid rule on a fine grid, give
    Z_deprot / Z_prot = 10^(pH - pKa)."""
    kT, h = 2.494339, 6.0
    d = lb.pfc_delta(pH=4.0 + dpH, pKa=4.0, h=h, kT=kT)
    assert _trapezoid_log10_ratio(0.0, 0.5, 1.0, h, d, kT) == pytest.approx(dpH, abs=2e-6)
    # deprotonated state favoured above the pKa: the lambda = 1 well is the lower one
    assert (d < 0) == (dpH > 0)


@pytest.mark.parametrize("dpH", [-1.5, 0.7])
def test_pfc_optional_bounds_over_the_walls(dpH):
    """The optional bounds (the reflecting walls -0.1 and 1.1) give the offset for which the
    sampled populations, walls included, have the Henderson-Hasselbalch ratio; it differs
    from the offset of the paper's [0, 1] integrals, since the walls' tails hold weight
    exp(-delta/kT) times larger on the deprotonated side."""
    kT, h = 2.494339, 6.0
    d = lb.pfc_delta(pH=4.0 + dpH, pKa=4.0, h=h, kT=kT, lo=-0.1, hi=1.1)
    assert _trapezoid_log10_ratio(-0.1, 0.5, 1.1, h, d, kT) == pytest.approx(dpH, abs=2e-6)
    d_paper = lb.pfc_delta(pH=4.0 + dpH, pKa=4.0, h=h, kT=kT)
    assert abs(d - d_paper) > 1e-3 * kT


@pytest.mark.parametrize("dpH,barrier", [(-1.5, 6.0), (0.0, 8.0), (0.7, 6.0), (2.0, 4.0)])
def test_library_pfc_matches_oracle(dpH, barrier):
    """The library's host-side correction (Gauss-Legendre, bisection) against the oracle's
    (adaptive quadrature, Brent)."""
    from paper_2410_01626_b300 import lambda_pfc
    kT = 2.494339
    want = lb.pfc_delta(pH=4.0 + dpH, pKa=4.0, h=barrier, kT=kT)
    got = lambda_pfc(4.0 + dpH, 4.0, barrier, kT)
    assert got == pytest.approx(want, abs=1e-9 * kT)
    # the optional bounds (the walls' interval) against the oracle with the same bounds
    want = lb.pfc_delta(pH=4.0 + dpH, pKa=4.0, h=barrier, kT=kT, lo=-0.1, hi=1.1)
    got = lambda_pfc(4.0 + dpH, 4.0, barrier, kT, lo=-0.1, hi=1.1)
    assert got == pytest.approx(want, abs=1e-9 * kT)


def test_library_pfc_rejects_bad_arguments():
    from paper_2410_01626_b300 import FmmError, lambda_pfc
    with pytest.raises(FmmError):
        lambda_pfc(7.0, 4.0, 5.0, kT=0.0)
    with pytest.raises(FmmError):
        lambda_pfc(7.0, 4.0, 5.0, a0=1.0, a1=0.0)
    with pytest.raises(FmmError):
        lambda_pfc(7.0, 4.0, 5.0, lo=0.6)  # an empty protonated interval
