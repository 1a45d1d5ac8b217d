"""Lambda-side potentials of the constant-pH Hamiltonian -- TEST INFRASTRUCTURE ONLY.

Plain FP64 restatement (only ``tests/`` may import it) of the bias potential on a lambda
coordinate (arXiv 2410.01626, Sec. 2.2 "Calibration of Protonation Dynamics"):

* the double well V_dw (cubic Hermite splines, Sec. 2.2): wells at a0 and a1, the central
  barrier at b = (a0 + a1) / 2, V(a0) = 0, V(b) = h, V(a1) = delta, zero slope at all three
  (so each piece is V_a + (V_b - V_a)(3 s^2 - 2 s^3)), and harmonic walls
  V = V(a0) + kw (l - a0)^2 / 2 below a0 and V(a1) + kw (l - a1)^2 / 2 above a1;
* the pH potential (Eq. 4): the free energy of deprotonation (lambda = 1 against 0) is
  ln(10) kT (pKa_ref - pH);
* the partition function correction (Sec. 2.3): the well offset delta is refined until the
  populations of the two states that V implies match that free energy, i.e.
  Z_deprot / Z_prot = 10^(pH - pKa_ref) with Z_prot = int_0^0.5 exp(-V/kT) and
  Z_deprot = int_0.5^1 exp(-V/kT), the bounds Sec. 2.3 states (lo = 0, hi = 1, split at the
  barrier b = 0.5 of the wells at 0 and 1).  Other bounds are an option: lo, hi = the
  reflecting walls (-0.1, 1.1) make the condition hold for the population the dynamics
  samples, a departure from the paper's integrals used only where a test needs that
  population.

Parity pins (tests/test_lambda_bias.py): the spline's values and slopes at the knots,
continuity, the symmetric case (pH = pKa, symmetric wells: delta = 0), and the population
ratio of the corrected potential by an independent quadrature over [0, 0.5] and [0.5, 1]
(and over the walls' interval for the optional bounds).
"""
from __future__ import annotations

import math

from scipy import integrate, optimize


def potential(l, a0, a1, h, delta, kw):
    """V_dw(l) and dV/dl."""
    b = 0.5 * (a0 + a1)
    if l < a0:
        return 0.5 * kw * (l - a0) ** 2, kw * (l - a0)
    if l > a1:
        return delta + 0.5 * kw * (l - a1) ** 2, kw * (l - a1)
    if l <= b:
        va, vb, la, lb = 0.0, h, a0, b
    else:
        va, vb, la, lb = h, delta, b, a1
    s = (l - la) / (lb - la)
    return va + (vb - va) * (3 * s * s - 2 * s ** 3), (vb - va) * (6 * s - 6 * s * s) / (lb - la)


def population_ratio(a0, a1, h, delta, kw, kT, lo=0.0, hi=1.0):
    """Z_deprot / Z_prot of exp(-V/kT) on [lo, hi] split at the barrier (Sec. 2.3: [0, 0.5]
    and [0.5, 1] by default)."""
    b = 0.5 * (a0 + a1)
    f = lambda l: math.exp(-potential(l, a0, a1, h, delta, kw)[0] / kT)  # noqa: E731
    pts = [a0, a1]
    zp = integrate.quad(f, lo, b, points=[p for p in pts if lo < p < b], epsabs=0, epsrel=1e-12, limit=200)[0]
    zd = integrate.quad(f, b, hi, points=[p for p in pts if b < p < hi], epsabs=0, epsrel=1e-12, limit=200)[0]
    return zd / zp


def pfc_delta(pH, pKa, h, kT, a0=0.0, a1=1.0, kw=1000.0, lo=0.0, hi=1.0):
    """The well offset delta for which Z_deprot / Z_prot = 10^(pH - pKa), the partition
    functions taken over [lo, b] and [b, hi] (Sec. 2.3: lo = 0, hi = 1)."""
    target = math.log(10.0) * (pH - pKa)
    g = lambda d: math.log(population_ratio(a0, a1, h, d, kw, kT, lo, hi)) - target  # noqa: E731
    lo_d, hi_d = -50 * kT - abs(target) * kT, 50 * kT + abs(target) * kT
    return optimize.brentq(g, lo_d, hi_d, xtol=1e-13, rtol=1e-14, maxiter=500)
