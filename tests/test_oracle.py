"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test checks the oracle against something other than itself: a closed
form (two charges, NaCl Madelung constant, Wigner constant of a single charge
in a neutralising background, the large-box limit of the tinfoil Ewald sum),
an invariant (Newton's third law, exact quadratic dependence on lambda,
alpha independence), finite differences, or brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

KE = oracle.KE_DEFAULT
_GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "constants.json")))
MADELUNG_NACL = _GOLD["madelung_nacl"]["value"]  # rock salt, nearest-neighbour distance
WIGNER_SC = _GOLD["wigner_simple_cubic"]["value"]  # simple cubic lattice with neutralising background


def test_two_charges_closed_form():
    x = np.array([[0.1, 0.2, 0.3], [0.4, -0.2, 0.9]])
    q = np.array([1.5, -0.7])
    phi, grad = oracle.direct(x, q)
    r = np.linalg.norm(x[0] - x[1])
    assert phi[0] == pytest.approx(q[1] / r, rel=1e-14)
    assert phi[1] == pytest.approx(q[0] / r, rel=1e-14)
    # force on 0: k q0 q1 (x0 - x1) / r^3
    F0 = -q[0] * grad[0]
    np.testing.assert_allclose(F0, q[0] * q[1] * (x[0] - x[1]) / r ** 3, rtol=1e-13)
    E = 0.5 * np.dot(q, phi)
    assert E == pytest.approx(q[0] * q[1] / r, rel=1e-14)


def test_direct_brute_force_pairs():
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 2, (7, 3))
    q = rng.normal(size=7)
    phi, _ = oracle.direct(x, q)
    E_pairs = sum(q[i] * q[j] / np.linalg.norm(x[i] - x[j]) for i in range(7) for j in range(i))
    assert 0.5 * np.dot(q, phi) == pytest.approx(E_pairs, rel=1e-13)


def test_direct_newton_and_fd_in_x():
    s = synth.open_uniform(seed=3, n=60, L=2.0, n_sites=3, site_size=4)
    x = s["x"].astype(np.float64)
    q, _ = oracle.charges(s["qA"], s["qB"], s["site"], s["lam"])
    phi, grad = oracle.direct(x, q)
    F = -q[:, None] * grad
    assert np.abs(F.sum(0)).max() < 1e-11 * np.abs(F).max()

    def energy(xx):
        p, _ = oracle.direct(xx, q)
        return 0.5 * np.dot(q, p)

    h = 1e-5
    for i in (0, 17, 42):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            fd = -(energy(xp) - energy(xm)) / (2 * h)
            assert fd == pytest.approx(F[i, a], rel=1e-6, abs=1e-8 * np.abs(F).max())


def test_charges_interpolation():
    qA = np.array([0.5, -0.25, 1.0], np.float32)
    qB = np.array([-0.5, 0.75, 3.0], np.float32)
    site = np.array([0, 1, -1], np.int32)
    lam = np.array([0.25, 1.0], np.float32)
    q, dq = oracle.charges(qA, qB, site, lam)
    np.testing.assert_allclose(q, [0.25, 0.75, 1.0], rtol=0, atol=0)
    np.testing.assert_allclose(dq, [-1.0, 1.0, 0.0], rtol=0, atol=0)


@pytest.mark.parametrize("periodic", [False, True])
def test_dvdlambda_is_exact_derivative(periodic):
    """E is exactly quadratic in each lambda_k, so the central difference is exact."""
    if periodic:
        s = synth.periodic_uniform(seed=5, n=40, L=1.5, n_sites=3, site_size=4)
    else:
        s = synth.open_uniform(seed=5, n=40, L=1.5, n_sites=3, site_size=4)
    out = oracle.evaluate(s, tol=1e-13)
    h = 1e-3
    for k in range(len(s["lam"])):
        lp = s["lam"].astype(np.float64).copy(); lp[k] += h
        lm = s["lam"].astype(np.float64).copy(); lm[k] -= h
        # evaluate with FP64 lambdas (FP32 cast would perturb h)
        def E_of(lam):
            x = s["x"].astype(np.float64)
            qA = s["qA"].astype(np.float64); qB = s["qB"].astype(np.float64)
            lam_i = np.where(s["site"] >= 0, lam[np.maximum(s["site"], 0)], 0.0)
            q = qA + lam_i * (qB - qA)
            if periodic:
                phi, _ = oracle.ewald(x, q, s["L"], tol=1e-13)
            else:
                phi, _ = oracle.direct(x, q)
            return 0.5 * KE * np.dot(q, phi)
        fd = (E_of(lp) - E_of(lm)) / (2 * h)
        assert fd == pytest.approx(out["dVdl"][k], rel=1e-8, abs=1e-9)


def _nacl(ncell, a):
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    na = []
    for i in range(ncell):
        for j in range(ncell):
            for k in range(ncell):
                na.append(base + [i, j, k])
    na = np.concatenate(na) * a
    cl = na + np.array([0.5, 0, 0]) * a
    x = np.concatenate([na, cl])
    q = np.concatenate([np.ones(len(na)), -np.ones(len(cl))])
    return x, q


def test_ewald_nacl_madelung():
    a = 0.5640
    x, q = _nacl(2, a)  # 64 ions, box 2a
    L = 2 * a
    phi, _ = oracle.ewald(x, q, L, tol=1e-13)
    d = a / 2
    M = -q * phi * d  # each ion: q_i phi_i = -M / d
    # the constant is quoted to six decimals: agree within half a unit of the last one
    np.testing.assert_allclose(M, MADELUNG_NACL, rtol=0, atol=5e-7)


@pytest.mark.parametrize("L", [1.0, 3.7])
def test_ewald_wigner_single_charge(L):
    x = np.array([[0.3 * L, 0.1 * L, 0.77 * L]])
    q = np.array([1.0])
    phi, grad = oracle.ewald(x, q, L, tol=1e-14)
    # xi is quoted to six decimals: agree within half a unit of the last one
    assert q[0] * phi[0] * L == pytest.approx(WIGNER_SC, abs=5e-7)
    assert np.abs(grad).max() < 1e-10 / L ** 2


def test_ewald_alpha_independence():
    s = synth.periodic_uniform(seed=9, n=50, L=2.0, n_sites=2, site_size=4, neutral=False)
    x = s["x"].astype(np.float64)
    q, _ = oracle.charges(s["qA"], s["qB"], s["site"], s["lam"])
    p1, g1 = oracle.ewald(x, q, 2.0, alpha=4.0, rc=1.6, mmax=14)
    p2, g2 = oracle.ewald(x, q, 2.0, alpha=6.5, rc=1.0, mmax=22)
    np.testing.assert_allclose(p1, p2, rtol=0, atol=1e-9 * np.abs(p1).max())
    np.testing.assert_allclose(g1, g2, rtol=0, atol=1e-9 * np.abs(g1).max())


@pytest.mark.parametrize("neutral", [True, False])
def test_ewald_large_box_limit(neutral):
    """A small cluster in a large periodic box: the tinfoil Ewald energy is
    E_direct + Q^2 xi / (2L) + (2 pi / 3V)(Q sum q|x-c|^2 - |D|^2) + O(s^4/L^5)
    (images beyond the central cell expanded to second order; the dipolar
    lattice sum vanishes by cubic symmetry, the neutralising background and the
    conducting boundary give the quadratic term)."""
    rng = np.random.default_rng(21)
    n = 12
    L = 25.0
    c = np.array([L / 2] * 3)
    x = c + rng.uniform(-0.5, 0.5, (n, 3))
    q = rng.normal(size=n)
    if neutral:
        q -= q.mean()
    phi_e, grad_e = oracle.ewald(x, q, L, tol=1e-14)
    phi_d, grad_d = oracle.direct(x, q)
    V = L ** 3
    Q = q.sum(); u = x - c; D = (q[:, None] * u).sum(0); T = (q * (u * u).sum(1)).sum()
    E_pred = 0.5 * np.dot(q, phi_d) + 0.5 * Q * Q * WIGNER_SC / L + 2 * math.pi / (3 * V) * (Q * T - D @ D)
    E_ew = 0.5 * np.dot(q, phi_e)
    assert E_ew == pytest.approx(E_pred, abs=2e-7 * abs(E_pred) + 1e-9)
    # forces: the same expansion gives grad phi_i = grad_direct + (4 pi/3V)(Q u_i - D)
    g_corr = 4 * math.pi / (3 * V) * (Q * u - D)
    g_pred = grad_d + g_corr
    # the neglected fourth-order lattice term moves the field by O(s^3/L^5), about 1e-6
    # here; a dropped or mis-signed quadratic term would miss by 100x that tolerance
    np.testing.assert_allclose(grad_e, g_pred, rtol=0, atol=1e-2 * np.abs(g_corr).max())
    # the tinfoil term is resolved by this check: it is much larger than the tolerance
    assert 2 * math.pi / (3 * V) * (D @ D) > 50 * 2e-7 * abs(E_pred)


def test_ewald_fd_in_x():
    s = synth.periodic_uniform(seed=13, n=30, L=1.2, n_sites=2, site_size=4, neutral=False)
    x = s["x"].astype(np.float64)
    q, _ = oracle.charges(s["qA"], s["qB"], s["site"], s["lam"])
    _, grad = oracle.ewald(x, q, 1.2, tol=1e-13)
    F = -q[:, None] * grad

    def energy(xx):
        p, _ = oracle.ewald(xx, q, 1.2, tol=1e-13)
        return 0.5 * np.dot(q, p)

    h = 1e-5
    for i in (0, 11, 29):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            fd = -(energy(xp) - energy(xm)) / (2 * h)
            assert fd == pytest.approx(F[i, a], rel=1e-5, abs=1e-7 * np.abs(F).max())
    # periodicity: moving an atom by a box vector changes nothing
    xs = x.copy(); xs[3] += np.array([1.2, -2.4, 0.0])
    assert energy(xs) == pytest.approx(energy(x), rel=1e-11)


def _bin_bruteforce(x, origin, L, depth, periodic):
    nb = 1 << depth
    s = math.ldexp(1.0, depth) / L
    n = len(x)
    key = np.zeros(n, np.uint64)
    st = 0
    for i in range(n):
        c = []
        for a in range(3):
            u = float(np.float64(x[i, a])) - origin[a]
            if periodic:
                u = u - L * math.floor(u / L)
                if u < 0.0 or u >= L:
                    u = 0.0
            elif not (0.0 <= u <= L):
                st |= 1
            f = math.floor(u * s)
            c.append(min(max(int(f), 0), nb - 1))
        k = 0
        for b in range(depth):
            for a in range(3):
                k |= ((c[a] >> b) & 1) << (3 * b + a)
        key[i] = k
    perm = np.argsort(key, kind="stable")
    count = np.bincount(key.astype(np.int64), minlength=1 << (3 * depth))
    start = np.concatenate([[0], np.cumsum(count)[:-1]])
    return key, perm, start, count, st


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("depth", [0, 1, 3])
def test_binning_bruteforce(periodic, depth):
    rng = np.random.default_rng(depth + 10 * periodic)
    L = 2.5
    origin = (-0.5, 0.25, 1.0)
    x = (np.array(origin) + rng.uniform(0, L, (300, 3))).astype(np.float32)
    # adversarial positions: on the faces, at origin + L, on leaf boundaries
    x[0] = origin
    x[1] = np.array(origin) + L
    x[2] = np.array(origin) + L / 2
    x[3] = np.array(origin) + [L / 8, L / 4, 3 * L / 8]
    if periodic:
        x[4] = np.array(origin) - [1e-7, 3 * L, 7.3 * L]
        x[5] = np.array(origin) + [2 * L, -L, L * 1.5]
    got = oracle.binning(x, origin, L, depth, periodic)
    ref = _bin_bruteforce(x, origin, L, depth, periodic)
    for g, r in zip(got[:4], ref[:4]):
        np.testing.assert_array_equal(g.astype(np.int64), np.asarray(r).astype(np.int64))
    assert got[4] == ref[4] == 0


def test_binning_open_domain_flag():
    x = np.array([[0.5, 0.5, 0.5], [1.2, 0.5, 0.5]], np.float32)
    *_, st = oracle.binning(x, (0, 0, 0), 1.0, 2, False)
    assert st == 1


# ---------------------------------------------------------------- pair potential (Hamiltonian form)
XI = -2.8372974794  # Wigner constant of the simple cubic lattice with background


@pytest.mark.parametrize("L", [1.0, 2.5, 7.0])
def test_pair_self_term_is_wigner(L):
    assert oracle.self_potential(L, True) * L == pytest.approx(XI, abs=1e-9)
    assert oracle.self_potential(None, False) == 0.0


def test_pair_potential_small_r_expansion_and_periodicity():
    """psi(r) = 1/r + xi/L + (2 pi / 3V) r^2 + O(r^4 / L^5) (degree 2 and odd harmonic
    terms vanish by cubic symmetry), and psi is periodic."""
    L = 2.0
    rng = np.random.default_rng(1)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        for s in (0.02, 0.05):
            r = s * L * d
            psi, _ = oracle.pair_potential(r, L, True)
            approx = 1.0 / np.linalg.norm(r) + XI / L + 2 * np.pi / (3 * L ** 3) * np.dot(r, r)
            assert abs(psi - approx) < 40.0 * s ** 4 / L
        r = rng.uniform(-0.5, 0.5, 3) * L
        for shift in (np.array([L, 0, 0]), np.array([0, -L, L])):
            assert oracle.pair_potential(r + shift, L, True)[0] == pytest.approx(oracle.pair_potential(r, L, True)[0],
                                                                                 abs=1e-9)


@pytest.mark.parametrize("periodic", [False, True])
def test_pair_potential_gradient_by_finite_differences(periodic):
    L = 3.0
    r = np.array([0.41, -0.27, 0.33])
    _, g = oracle.pair_potential(r, L, periodic)
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (oracle.pair_potential(r + e, L, periodic)[0] - oracle.pair_potential(r - e, L, periodic)[0]) / (2 * h)
        assert fd == pytest.approx(g[a], rel=1e-6, abs=1e-9)


def _two_site_system(periodic):
    if periodic:
        s = synth.periodic_uniform(seed=14, n=80, L=2.2, n_sites=2, site_size=4, neutral=False, p=6, depth=1)
    else:
        s = synth.open_uniform(seed=14, n=80, L=2.2, n_sites=2, site_size=4, p=6, depth=1)
    return s


def _energy(s, lam, hamiltonian):
    t = dict(s)
    t["lam"] = np.asarray(lam, np.float32)
    return oracle.evaluate(t, tol=1e-12, hamiltonian=hamiltonian)


@pytest.mark.parametrize("periodic", [False, True])
def test_hamiltonian_form_is_multilinear_in_lambda(periodic):
    """Interpolating the Hamiltonian makes E linear in each site lambda; at lambda_k in
    {0, 1} it equals the charge-interpolated energy.  So E_H(l1, l2) is the bilinear
    interpolation of the four corner energies of the (pinned) charge form, and
    dE_H/dl_k is the corner difference."""
    s = _two_site_system(periodic)
    corner = {(a, b): _energy(s, [a, b], False)["E"] for a in (0.0, 1.0) for b in (0.0, 1.0)}
    l1, l2 = 0.375, 0.8125  # exact in FP32, the precision of the lambda inputs
    out = _energy(s, [l1, l2], True)
    bil = ((1 - l1) * (1 - l2) * corner[0, 0] + l1 * (1 - l2) * corner[1, 0] + (1 - l1) * l2 * corner[0, 1]
           + l1 * l2 * corner[1, 1])
    scale = max(abs(v) for v in corner.values())
    assert out["E"] == pytest.approx(bil, abs=1e-9 * scale)
    d1 = (1 - l2) * (corner[1, 0] - corner[0, 0]) + l2 * (corner[1, 1] - corner[0, 1])
    d2 = (1 - l1) * (corner[0, 1] - corner[0, 0]) + l1 * (corner[1, 1] - corner[1, 0])
    assert out["dVdl"][0] == pytest.approx(d1, abs=1e-9 * scale)
    assert out["dVdl"][1] == pytest.approx(d2, abs=1e-9 * scale)
    # and it differs from the charge form away from the corners
    assert abs(out["E"] - _energy(s, [l1, l2], False)["E"]) > 1e-6 * scale


@pytest.mark.parametrize("periodic", [False, True])
def test_hamiltonian_forces_by_finite_differences(periodic):
    s = _two_site_system(periodic)
    lam = [0.375, 0.625]
    out = _energy(s, lam, True)
    site_atoms = np.nonzero(s["site"] >= 0)[0][:3]
    h = 1e-4
    for i in site_atoms:
        for a in range(3):
            xp = s["x"].astype(np.float64).copy()
            xm = xp.copy()
            xp[i, a] += h
            xm[i, a] -= h
            sp, sm = dict(s), dict(s)
            sp["x"], sm["x"] = xp, xm
            # positions are FP32 inputs: difference over the step the rounded coordinates take
            h_eff = (float(np.float32(xp[i, a])) - float(np.float32(xm[i, a]))) / 2
            fd = -(_energy(sp, lam, True)["E"] - _energy(sm, lam, True)["E"]) / (2 * h_eff)
            assert fd == pytest.approx(out["F"][i, a], rel=1e-5, abs=1e-6 * np.abs(out["F"]).max())


# ---------------------------------------------------------------- four-form sites (Eq. 2)
def _four_form_system(periodic, tautomer_fraction=1.0):
    return synth.tautomer_sites(_two_site_system(periodic), seed=3, tautomer_fraction=tautomer_fraction)


def _energy4(s, lam2, hamiltonian):
    t = dict(s)
    t["lam"] = np.asarray(lam2, np.float32)
    return oracle.evaluate(t, tol=1e-12, hamiltonian=hamiltonian)


@pytest.mark.parametrize("periodic", [False, True])
def test_four_form_hamiltonian_is_multilinear(periodic):
    """Eq. 2 makes E linear in each of the four coordinates (lp, lt of two sites): E_H
    equals the multilinear interpolation of the sixteen corner energies, where every site
    is in one pure form and both interpolations agree; dE/dl is the matching difference."""
    import itertools
    s = _four_form_system(periodic)
    lam = np.array([0.375, 0.8125, 0.625, 0.25])  # exact in FP32
    corners = {c: _energy4(s, np.array(c, float), False)["E"] for c in itertools.product((0.0, 1.0), repeat=4)}
    out = _energy4(s, lam, True)

    def interp(l):
        return sum(np.prod([li if ci else 1 - li for ci, li in zip(c, l)]) * e for c, e in corners.items())

    scale = max(abs(v) for v in corners.values())
    assert out["E"] == pytest.approx(interp(lam), abs=1e-10 * scale)
    for j in range(4):  # dE/dl_j of a multilinear function: interpolation of the corner differences
        lo, hi = lam.copy(), lam.copy()
        lo[j], hi[j] = 0.0, 1.0
        assert out["dVdl"][j] == pytest.approx(interp(hi) - interp(lo), abs=1e-10 * scale)
    assert abs(out["E"] - _energy4(s, lam, False)["E"]) > 1e-6 * scale


@pytest.mark.parametrize("periodic", [False, True])
def test_four_form_charge_derivatives_by_finite_differences(periodic):
    """Charge interpolation: E is quadratic in each coordinate, so central differences
    are exact up to rounding."""
    s = _four_form_system(periodic)
    lam = np.array([0.375, 0.8125, 0.625, 0.25])
    out = _energy4(s, lam, False)
    h = 0.125
    for j in range(4):
        lp, lm = lam.copy(), lam.copy()
        lp[j] += h
        lm[j] -= h
        fd = (_energy4(s, lp, False)["E"] - _energy4(s, lm, False)["E"]) / (2 * h)
        assert fd == pytest.approx(out["dVdl"][j], rel=1e-9, abs=1e-9 * abs(out["E"]))


@pytest.mark.parametrize("hamiltonian", [False, True])
def test_four_form_reduces_to_two_forms(hamiltonian):
    """Sites without tautomers (qB = qA, qD = qC) are the two-form sites of Eq. 1 with
    lambda = lp; their lt derivative vanishes."""
    s2 = _two_site_system(True)
    s4 = _four_form_system(True, tautomer_fraction=0.0)
    lam4 = np.array([0.375, 0.8125, 0.625, 0.25])
    a = _energy4(s4, lam4, hamiltonian)
    b = _energy(s2, lam4[0::2], hamiltonian)
    assert a["E"] == pytest.approx(b["E"], rel=1e-12)
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-9, atol=1e-9 * np.abs(b["F"]).max())
    np.testing.assert_allclose(a["dVdl"][0::2], b["dVdl"], rtol=1e-9)
    assert np.abs(a["dVdl"][1::2]).max() < 1e-9 * np.abs(b["dVdl"]).max()


def test_four_form_hamiltonian_forces_by_finite_differences():
    s = _four_form_system(True)
    lam = np.array([0.375, 0.8125, 0.625, 0.25])
    out = _energy4(s, lam, True)
    h = 1e-4
    for i in np.nonzero(s["site"] >= 0)[0][:2]:
        for a in range(3):
            xp = s["x"].astype(np.float64).copy()
            xm = xp.copy()
            xp[i, a] += h
            xm[i, a] -= h
            sp, sm = dict(s), dict(s)
            sp["x"], sm["x"] = xp, xm
            h_eff = (float(np.float32(xp[i, a])) - float(np.float32(xm[i, a]))) / 2
            fd = -(_energy4(sp, lam, True)["E"] - _energy4(sm, lam, True)["E"]) / (2 * h_eff)
            assert fd == pytest.approx(out["F"][i, a], rel=1e-5, abs=1e-6 * np.abs(out["F"]).max())
