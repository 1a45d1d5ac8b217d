"""Oracle for the FMM constant-pH electrostatics path -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU restatement of what the GPU fast multipole method
approximates.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg may import it.  It shares no code with the CUDA path
(``paper_2410_01626_b300``): it neither imports that package nor is imported
by it.

What it computes (citations are to arXiv 2410.01626):

* ``charges``: q_i = qA_i + lambda_{s(i)} (qB_i - qA_i), dq_i = qB_i - qA_i
  (Sec. 2.1, Eq. 1: the Hamiltonian is interpolated linearly in lambda, and
  the protonated and deprotonated forms differ only in their charges).  Atoms
  outside every site keep q_i = qA_i.
* ``direct``: open-boundary Coulomb potential phi_i = sum_{j != i} q_j / r_ij
  and its gradient (the quantity the FMM solver of Sec. 2.6 approximates).
* ``ewald``: the same for a periodic cube with tinfoil boundary and uniform
  neutralising background, phi_i = dE_Ewald / dq_i.
* ``evaluate``: E = 1/2 k_e sum q_i phi_i, F_i = -k_e q_i grad phi_i and
  dV/dlambda_k = k_e sum_{i in site k} dq_i phi_i (E is quadratic in the
  charges, so dE/dq_i = k_e phi_i; the chain rule through q_i(lambda) gives
  the site derivative that drives the lambda particle, Sec. 2.1).
* ``binning``: the Morton-key leaf binning specification (keys, stable
  permutation, leaf ranges).
* ``charges4`` / four-form systems (``forms`` = 4): sites with two lambda
  coordinates over four charge forms (Sec. 2.1, Eq. 2), dV/dlambda per site
  and coordinate; ``hamiltonian_correction4`` the Hamiltonian form of them.
* ``pair_potential`` / ``self_potential``: the pair potential psi(r) of the
  energy above (1/r open; the Ewald pair potential periodic) and its
  self-image limit psi_0 (0 open; xi / L periodic).
* ``hamiltonian_correction``: the difference between interpolating the
  Hamiltonian and interpolating the charges (Sec. 2.1, Eq. 1).  For atoms i, j
  of one site k, (1 - lambda) qA_i qA_j + lambda qB_i qB_j - q_i(lambda) q_j(lambda)
  = lambda (1 - lambda) dq_i dq_j, and pairs in different sites agree in both
  forms, so E_H - E_q = k_e sum_k lambda_k (1 - lambda_k) [sum_{i<j in k}
  dq_i dq_j psi(r_ij) + 1/2 sum_{i in k} dq_i^2 psi_0].  ``evaluate(...,
  hamiltonian=True)`` adds it and its derivatives.

Pins (tests/test_oracle.py): two-charge closed form, NaCl Madelung constant,
Wigner constant of a single charge with background, alpha independence, the
de Leeuw-Perram-Smith tinfoil/vacuum relation, finite differences in x and
lambda, brute-force binning on tiny inputs; for the pair potential the Wigner
constant (psi_0 L = xi), the small-r expansion 1/r + xi/L + (2 pi / 3V) r^2 and
periodicity; for the Hamiltonian form, multilinearity in the site lambdas
(the energy at any lambda is the multilinear interpolation of the
charge-interpolated energies at lambda_k in {0, 1}, where the two forms agree).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import time

import numpy as np

KE_DEFAULT = 138.935458  # kJ mol^-1 nm e^-2 (GROMACS unit system)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (FP64, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.orc_charges.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P, P, P]
        _lib.orc_direct.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P]
        _lib.orc_ewald.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P]
        _lib.orc_bin.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 P, P, P, P, P]
        _lib.orc_nthreads.restype = ctypes.c_int
        _lib.orc_ewald_phase_seconds.argtypes = [P]
        _lib.orc_ewald_pair.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def nthreads() -> int:
    return int(_load().orc_nthreads())


def ewald_phase_seconds():
    """Wall-clock seconds of the last Ewald call's two phases: (structure factors, per-target
    sums).  Timing only, for the CPU baseline."""
    out = np.zeros(2)
    _load().orc_ewald_phase_seconds(_p(out))
    return float(out[0]), float(out[1])


def charges(qA, qB, site, lam):
    """q_i and dq_i in FP64 from FP32 inputs (Sec. 2.1, Eq. 1)."""
    qA = np.ascontiguousarray(qA, np.float32)
    qB = np.ascontiguousarray(qB, np.float32)
    site = np.ascontiguousarray(site, np.int32)
    lam = np.ascontiguousarray(lam, np.float32)
    n = len(qA)
    q = np.empty(n)
    dq = np.empty(n)
    _load().orc_charges(n, _p(qA), _p(qB), _p(site), len(lam), _p(lam), _p(q), _p(dq))
    return q, dq


def charges4(qA, qB, qC, qD, site, lam2):
    """Sites with two lambda coordinates (Sec. 2.1, Eq. 2): with lp, lt of the atom's site,
    q_i = (1 - lp)[(1 - lt) qA_i + lt qB_i] + lp[(1 - lt) qC_i + lt qD_i] (FP64 from FP32
    inputs), and the derivatives dq/dlp, dq/dlt.  lam2 = [2K]: (lp, lt) per site.  Atoms
    outside every site keep qA."""
    a, b, c, d = (np.asarray(v, np.float32).astype(np.float64) for v in (qA, qB, qC, qD))
    site = np.asarray(site, np.int64)
    l2 = np.asarray(lam2, np.float32).astype(np.float64).reshape(-1, 2)
    K = len(l2)
    ins = (site >= 0) & (site < K)
    k = np.where(ins, site, 0)
    p = np.where(ins, l2[k, 0] if K else 0.0, 0.0)
    t = np.where(ins, l2[k, 1] if K else 0.0, 0.0)
    q = np.where(ins, (1 - p) * ((1 - t) * a + t * b) + p * ((1 - t) * c + t * d), a)
    dqp = np.where(ins, ((1 - t) * c + t * d) - ((1 - t) * a + t * b), 0.0)
    dqt = np.where(ins, (1 - p) * (b - a) + p * (d - c), 0.0)
    return q, dqp, dqt


def _targets(targets, n):
    if targets is None:
        return None, n
    t = np.ascontiguousarray(targets, np.int32)
    return t, len(t)


def direct(x, q, targets=None):
    """Open-boundary potential and its gradient at the target atoms."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, np.float64)
    t, nt = _targets(targets, len(q))
    phi = np.empty(nt)
    grad = np.empty((nt, 3))
    _load().orc_direct(len(q), _p(x), _p(q), nt, None if t is None else _p(t), _p(phi), _p(grad))
    return phi, grad


def ewald_params(L, tol=1e-11, rc=None):
    """Splitting parameter, real cutoff and reciprocal index cutoff for a
    target relative truncation error ``tol`` (erfc(alpha rc) ~ tol and
    exp(-k^2/4alpha^2) ~ tol)."""
    s = math.sqrt(-math.log(tol))
    if rc is None:
        rc = 0.5 * L
    alpha = s / rc
    kmax = 2.0 * alpha * s
    mmax = int(math.ceil(kmax * L / (2.0 * math.pi)))
    return alpha, rc, mmax


def ewald(x, q, L, targets=None, tol=1e-11, alpha=None, rc=None, mmax=None):
    """Periodic potential (tinfoil, neutralising background) and its gradient."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, np.float64)
    a0, rc0, m0 = ewald_params(L, tol, rc)
    alpha = a0 if alpha is None else alpha
    rc = rc0 if rc is None else rc
    if mmax is None:
        mmax = int(math.ceil(2.0 * alpha * math.sqrt(-math.log(tol)) * L / (2.0 * math.pi)))
    t, nt = _targets(targets, len(q))
    phi = np.empty(nt)
    grad = np.empty((nt, 3))
    _load().orc_ewald(len(q), _p(x), _p(q), float(L), float(alpha), float(rc), int(mmax), nt,
                      None if t is None else _p(t), _p(phi), _p(grad))
    return phi, grad


def _pair(r, L, periodic, self_term, tol):
    if not periodic:
        if self_term:
            return 0.0, np.zeros(3)
        r = np.asarray(r, np.float64)
        d = float(np.sqrt(np.dot(r, r)))
        return 1.0 / d, -r / d ** 3
    alpha, rc, mmax = ewald_params(L, tol)
    rr = np.ascontiguousarray(np.zeros(3) if r is None else r, np.float64)
    psi = np.zeros(1)
    grad = np.zeros(3)
    _load().orc_ewald_pair(_p(rr), int(bool(self_term)), float(L), float(alpha), float(rc), int(mmax), _p(psi),
                           _p(grad))
    return float(psi[0]), grad


def pair_potential(r, L=None, periodic=False, tol=1e-11):
    """psi(r) and d psi / d r for displacement r (unit charges, k_e = 1)."""
    return _pair(r, L, periodic, False, tol)


def self_potential(L=None, periodic=False, tol=1e-11):
    """psi_0 = lim_{r -> 0} (psi(r) - 1/|r|): 0 open, xi / L periodic."""
    return _pair(None, L, periodic, True, tol)[0]


def hamiltonian_correction(sys_, ke=KE_DEFAULT, tol=1e-11):
    """E_H - E_q and its derivatives for a system dict: returns E (float), F [n,3]
    (-dE/dx), dVdl [K] (dE/dlambda), phi_h [n] (dE/d dq_i = ke lambda (1 - lambda) phi_h_i)."""
    x = np.asarray(sys_["x"], np.float32).astype(np.float64)
    _, dq = charges(sys_["qA"], sys_["qB"], sys_["site"], sys_["lam"])
    site = np.asarray(sys_["site"], np.int64)
    lam = np.asarray(sys_["lam"], np.float32).astype(np.float64)
    L, periodic = sys_["L"], bool(sys_["periodic"])
    n, K = len(dq), len(lam)
    F = np.zeros((n, 3))
    phi_h = np.zeros(n)
    dvdl = np.zeros(K)
    E = 0.0
    psi0 = self_potential(L, periodic, tol)
    for k in range(K):
        atoms = np.nonzero(site == k)[0]
        w = lam[k] * (1.0 - lam[k])
        e_site = 0.0
        for a in atoms:
            phi_h[a] += dq[a] * psi0
            e_site += 0.5 * dq[a] ** 2 * psi0
        for ia, a in enumerate(atoms):
            for b in atoms[ia + 1:]:
                r = x[a] - x[b]
                if periodic:
                    r = r - L * np.round(r / L)
                psi, g = pair_potential(r, L, periodic, tol)
                e_site += dq[a] * dq[b] * psi
                phi_h[a] += dq[b] * psi
                phi_h[b] += dq[a] * psi
                F[a] -= ke * w * dq[a] * dq[b] * g
                F[b] += ke * w * dq[a] * dq[b] * g
        E += ke * w * e_site
        dvdl[k] = ke * (1.0 - 2.0 * lam[k]) * e_site
    return {"E": E, "F": F, "dVdl": dvdl, "phi_h": phi_h}


def hamiltonian_correction4(sys_, ke=KE_DEFAULT, tol=1e-11):
    """The Hamiltonian-interpolation correction for sites with four forms (Eq. 2).  With
    weights w_X(lp, lt) of the forms X in {A, B, C, D} and q_i = sum_X w_X q^X_i, the pair
    term of atoms i, j of one site changes by C_ij = sum_X w_X q^X_i q^X_j - q_i q_j
    = sum_X w_X (q^X_i - q_i)(q^X_j - q_j) (i = j with psi_0), and
    dC_ij/dl = sum_X (dw_X/dl)(q^X_i - q_i)(q^X_j - q_j).  Returns E, F [n,3],
    dVdl [2K] (lp, lt per site) and g_h [n,4]: dE/dq^X_i = ke w_X g_h[i, X]."""
    x = np.asarray(sys_["x"], np.float32).astype(np.float64)
    Q = np.stack([np.asarray(sys_[k], np.float32).astype(np.float64) for k in ("qA", "qB", "qC", "qD")], 1)
    q, _, _ = charges4(sys_["qA"], sys_["qB"], sys_["qC"], sys_["qD"], sys_["site"], sys_["lam"])
    site = np.asarray(sys_["site"], np.int64)
    l2 = np.asarray(sys_["lam"], np.float32).astype(np.float64).reshape(-1, 2)
    L, periodic = sys_["L"], bool(sys_["periodic"])
    n, K = len(q), len(l2)
    F = np.zeros((n, 3))
    g_h = np.zeros((n, 4))
    dvdl = np.zeros((K, 2))
    E = 0.0
    psi0 = self_potential(L, periodic, tol)
    for k in range(K):
        p, t = l2[k]
        w = np.array([(1 - p) * (1 - t), (1 - p) * t, p * (1 - t), p * t])
        wp = np.array([-(1 - t), -t, 1 - t, t])
        wt = np.array([-(1 - p), 1 - p, -p, p])
        atoms = np.nonzero(site == k)[0]
        dev = Q[atoms] - q[atoms, None]  # q^X_i - q_i
        for ia, a in enumerate(atoms):
            c = np.dot(w, dev[ia] ** 2)
            E += ke * 0.5 * c * psi0
            dvdl[k, 0] += ke * 0.5 * np.dot(wp, dev[ia] ** 2) * psi0
            dvdl[k, 1] += ke * 0.5 * np.dot(wt, dev[ia] ** 2) * psi0
            g_h[a] += dev[ia] * psi0
            for ib in range(ia + 1, len(atoms)):
                b = atoms[ib]
                r = x[a] - x[b]
                if periodic:
                    r = r - L * np.round(r / L)
                psi, g = pair_potential(r, L, periodic, tol)
                prod = dev[ia] * dev[ib]
                cab = np.dot(w, prod)
                E += ke * cab * psi
                dvdl[k, 0] += ke * np.dot(wp, prod) * psi
                dvdl[k, 1] += ke * np.dot(wt, prod) * psi
                F[a] -= ke * cab * g
                F[b] += ke * cab * g
                g_h[a] += dev[ib] * psi
                g_h[b] += dev[ia] * psi
    return {"E": E, "F": F, "dVdl": dvdl.reshape(-1), "g_h": g_h}


def evaluate(sys_, targets=None, ke=KE_DEFAULT, tol=1e-11, site_atoms=True, hamiltonian=False):
    """E, F, dV/dlambda for a synthetic system dict (keys of ``synth``); with
    ``hamiltonian`` the Hamiltonian-interpolation form (charge-interpolation
    energy plus ``hamiltonian_correction``).

    With ``targets`` given, phi/F are returned for those atoms only; E is then
    not computed (it needs every phi) and dV/dlambda is computed from the
    site atoms, which are added to the evaluated set when ``site_atoms``.
    """
    x = np.asarray(sys_["x"], np.float32).astype(np.float64)
    four = sys_.get("forms", 2) == 4
    if four:
        q, dq, dqt = charges4(sys_["qA"], sys_["qB"], sys_["qC"], sys_["qD"], sys_["site"], sys_["lam"])
        K = len(sys_["lam"]) // 2
    else:
        q, dq = charges(sys_["qA"], sys_["qB"], sys_["site"], sys_["lam"])
        K = len(sys_["lam"])
    n = len(q)
    site = np.asarray(sys_["site"], np.int64)
    if targets is None:
        idx = np.arange(n)
    else:
        idx = np.asarray(targets, np.int64)
        if site_atoms:
            idx = np.union1d(idx, np.nonzero(site >= 0)[0])
    t0 = time.perf_counter()
    if sys_["periodic"]:
        phi, grad = ewald(x, q, sys_["L"], None if targets is None else idx, tol=tol)
    else:
        phi, grad = direct(x, q, None if targets is None else idx)
    dt = time.perf_counter() - t0
    out = {"idx": idx, "phi": ke * phi, "F": -ke * q[idx, None] * grad, "seconds": dt}
    if targets is None:
        out["E"] = 0.5 * ke * float(np.dot(q, phi))
    dvdl = np.zeros(K)
    sel = site[idx] >= 0
    np.add.at(dvdl, site[idx][sel], dq[idx][sel] * phi[sel])
    out["dVdl"] = ke * dvdl
    if four:  # (dE/dlp, dE/dlt) per site, interleaved
        dvt = np.zeros(K)
        np.add.at(dvt, site[idx][sel], dqt[idx][sel] * phi[sel])
        out["dVdl"] = ke * np.stack([dvdl, dvt], 1).reshape(-1)
    if hamiltonian:
        h = hamiltonian_correction4(sys_, ke, tol) if four else hamiltonian_correction(sys_, ke, tol)
        out["F"] = out["F"] + h["F"][idx]
        out["dVdl"] = out["dVdl"] + h["dVdl"]
        if "E" in out:
            out["E"] += h["E"]
        if "phi_h" in h:
            out["phi_h"] = h["phi_h"][idx]
        if "g_h" in h:
            out["g_h"] = h["g_h"][idx]
    return out


def binning(x, origin, L, depth, periodic):
    """Binning specification: (key, perm, start, count, status)."""
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    n = len(x)
    o = np.ascontiguousarray(origin, np.float64)
    nleaf = 1 << (3 * depth)
    key = np.empty(n, np.uint32)
    perm = np.empty(n, np.uint32)
    start = np.empty(nleaf, np.uint32)
    count = np.empty(nleaf, np.uint32)
    st = np.zeros(1, np.int32)
    _load().orc_bin(n, _p(x), _p(o), float(L), int(depth), int(bool(periodic)), _p(key), _p(perm),
                    _p(start), _p(count), _p(st))
    return key, perm, start, count, int(st[0])
