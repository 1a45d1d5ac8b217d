"""CPU tests of the library's host logic: exports, operator construction, lattice operator.

No GPU is needed: the translation operators are built by the library's FP64
host code (fmm_host_operator) and checked against exact identities of the
multipole expansions, against direct Coulomb sums, and -- for the periodic
lattice operator -- against the oracle's Ewald potential.
"""
import itertools
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2410_01626_b300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "fmmcph.h")).read()
    declared = set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    lib = binding.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTS), declared ^ set(binding.EXPORTS)
    assert lib.fmm_build_flags() == 0


def test_bounds_checked_build_exports_every_declared_symbol():
    """The -DFMM_BOUNDS_CHECK variant (loaded by the tests with FMMCPH_BOUNDS_CHECK=1) has the
    same C ABI and says how it was built; no GPU call is made."""
    import ctypes
    path = binding._build.LIB_CHECKED
    if not os.path.exists(path):
        binding._build.build(checked=True)
    hdr = open(os.path.join(ROOT, "include", "fmmcph.h")).read()
    lib = ctypes.CDLL(path)
    for name in set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", hdr)):
        assert hasattr(lib, name), name
    lib.fmm_build_flags.restype = ctypes.c_int
    assert lib.fmm_build_flags() == 1


def _p2m(xs, qs, c, h, p):
    """Multipole of point charges with the library's basis (conj of Rhat)."""
    M = np.zeros((p + 1) ** 2)
    for x, q in zip(xs, qs):
        R = binding.host_regular(p, (x - c) / h)
        for n in range(p + 1):
            M[n * n] += q * R[n * n]
            for m in range(1, n + 1):
                M[n * n + 2 * m - 1] += q * R[n * n + 2 * m - 1]
                M[n * n + 2 * m] -= q * R[n * n + 2 * m]
    return M


def _l2p(L, x, c, h, p):
    R = binding.host_regular(p, (x - c) / h)
    s = 0.0
    for n in range(p + 1):
        s += L[n * n] * R[n * n]
        for m in range(1, n + 1):
            s += 2 * (L[n * n + 2 * m - 1] * R[n * n + 2 * m - 1] - L[n * n + 2 * m] * R[n * n + 2 * m])
    return s / h


@pytest.mark.parametrize("oct_", [0, 3, 5, 7])
def test_m2m_is_exact(oct_):
    p = 7
    rng = np.random.default_rng(oct_)
    hc = 0.5
    off = np.array([(oct_ >> a) & 1 for a in range(3)], float)
    cpar = np.array([1.0, 2.0, 3.0])
    cch = cpar + (off - 0.5) * hc
    xs = cch + rng.uniform(-hc / 2, hc / 2, (6, 3))
    qs = rng.normal(size=6)
    A = binding.host_operator(1, p, (oct_, 0, 0))
    np.testing.assert_allclose(A @ _p2m(xs, qs, cch, hc, p), _p2m(xs, qs, cpar, 2 * hc, p), atol=1e-13)


def test_l2l_is_exact():
    p = 6
    rng = np.random.default_rng(1)
    Lp = rng.normal(size=(p + 1) ** 2)
    for oct_ in range(8):
        B = binding.host_operator(2, p, (oct_, 0, 0))
        hc = 0.25
        cpar = np.zeros(3)
        cch = (np.array([(oct_ >> a) & 1 for a in range(3)]) - 0.5) * hc
        x = cch + rng.uniform(-hc / 2, hc / 2, 3)
        assert _l2p(B @ Lp, x, cch, hc, p) == pytest.approx(_l2p(Lp, x, cpar, 2 * hc, p), rel=1e-12)


def test_m2l_converges_to_direct_sum():
    rng = np.random.default_rng(4)
    h = 0.3
    o = (2, -3, 1)
    cs = np.array([0.15, 0.15, 0.15])
    ct = cs - np.array(o) * h
    xs = cs + rng.uniform(-h / 2, h / 2, (8, 3))
    qs = rng.normal(size=8)
    xt = ct + rng.uniform(-h / 2, h / 2, (5, 3))
    direct = np.array([sum(q / np.linalg.norm(x - s) for s, q in zip(xs, qs)) for x in xt])
    errs = []
    for p in (3, 5, 7, 9, 11):
        T = binding.host_operator(0, p, o)
        L = T @ _p2m(xs, qs, cs, h, p)
        fmm = np.array([_l2p(L, x, ct, h, p) for x in xt])
        errs.append(np.abs(fmm - direct).max() / np.abs(direct).max())
    assert errs[-1] < 1e-5
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def _lattice_h(p, r):
    lam = binding.host_operator(3, p)
    g = lam[:, 0]  # column 0: the harmonic coefficients of h in the normalised basis
    R = binding.host_regular(p, r)
    s = 0.0
    for n in range(p + 1):
        s += g[n * n] * R[n * n]
        for m in range(1, n + 1):
            s += 2 * (g[n * n + 2 * m - 1] * R[n * n + 2 * m - 1] - g[n * n + 2 * m] * R[n * n + 2 * m])
    return s


def test_lattice_operator_matches_ewald_remainder():
    """h(r) = psi_Ewald(r) - sum_{27 images} 1/|r - n| - (2 pi / 3)|r|^2 (unit cube)."""
    p = 12
    rng = np.random.default_rng(7)
    near = [np.array(n) for n in itertools.product((-1, 0, 1), repeat=3)]

    def h_ref(r):
        x = np.array([[0.5, 0.5, 0.5], 0.5 + r])
        phi, _ = oracle.ewald(x, np.array([1.0, 0.0]), 1.0, targets=[1], tol=1e-14)
        return phi[0] - sum(1.0 / np.linalg.norm(r - n) for n in near) - 2 * math.pi / 3 * (r @ r)

    for r in rng.normal(size=(6, 3)):
        r = 0.3 * r / np.linalg.norm(r)
        assert _lattice_h(p, r) == pytest.approx(h_ref(r), abs=2e-12)
    # farther out the truncated expansion converges geometrically in p
    r = np.array([0.5, 0.35, -0.2])
    ref = h_ref(r)
    errs = [abs(_lattice_h(q, r) - ref) for q in (6, 8, 10, 12, 14)]
    assert errs[-1] < 1e-8 and errs[-1] < errs[0] / 1000, errs


def test_lattice_constant_is_wigner_minus_near_images():
    lam = binding.host_operator(3, 8)
    near = 6 + 12 / math.sqrt(2) + 8 / math.sqrt(3)
    assert lam[0, 0] == pytest.approx(-2.837297 - near, abs=1e-6)
    # odd degrees and degree 2 vanish by cubic symmetry
    assert np.abs(lam[1:9, 0]).max() < 1e-12


def test_lattice_remainder_has_cubic_symmetry():
    rng = np.random.default_rng(3)
    for r in rng.uniform(-0.4, 0.4, (4, 3)):
        base = _lattice_h(10, r)
        for rr in (r[[1, 2, 0]], r * [-1, 1, 1], r[[0, 2, 1]] * [1, -1, 1]):
            assert _lattice_h(10, rr) == pytest.approx(base, abs=1e-12)


def test_argument_validation_on_host():
    with pytest.raises(binding.FmmError):
        binding.host_operator(0, 5, (1, 0, 0))   # a near-field offset has no M2L
    with pytest.raises(binding.FmmError):
        binding.host_operator(1, 0)               # p out of range
    with pytest.raises(binding.FmmError):
        binding.host_operator(7, 4)               # unknown kind
