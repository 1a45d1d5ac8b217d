"""Hamiltonian interpolation within sites (Sec. 2.1, Eq. 1) on the GPU.

The CUDA path adds lambda_k (1 - lambda_k) dq_i dq_j psi(r_ij) for every pair of one site
(and the self-image term) to the charge-interpolated FMM result.  Checked against the
FP64 oracle: the full E, F and dV/dlambda within the FMM tolerances, and the correction
alone -- the difference between a Hamiltonian-form and a charge-form handle, which share
the charge-form part bit for bit -- against the oracle's correction, at FP32 precision.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from fmm_check import errors, make_solver, oracle_ref, run_gpu, to_dev
from paper_2410_01626_b300 import fmm_energy

pytestmark = pytest.mark.gpu


def _systems():
    return [
        synth.open_uniform(seed=31, n=3000, L=4.0, n_sites=12, site_size=5, p=10, depth=3),
        synth.periodic_uniform(seed=32, n=3000, L=3.0, n_sites=12, site_size=5, neutral=False, p=10, depth=3),
        synth.solvated_30k(p=10),
    ]


@pytest.mark.parametrize("which,precision", [(0, "fp32"), (1, "fp32"), (2, "fp32"), (0, "3xtf32"), (1, "3xtf32"),
                                             (2, "3xtf32"), (0, "3xbf16"), (2, "3xbf16"), (0, "fp16"),
                                             (1, "fp16"), (2, "fp16")])
def test_hamiltonian_parity_with_oracle(which, precision):
    s = _systems()[which]
    tg = None if which < 2 else np.arange(0, len(s["x"]), 97)
    ref = oracle_ref(s, targets=tg, hamiltonian=True, tol=1e-10)
    g = run_gpu(s, precision=precision, interpolation="hamiltonian")
    e = errors(g, ref, idx=ref["idx"] if tg is not None else None)
    assert g["status"] == 0
    assert e["F"] < 1e-4 and e["dVdl"] < 1e-4, e
    if "E" in e:
        assert e["E"] < 1e-4, e


def test_hamiltonian_adds_no_error_in_split_bf16():
    """On the small non-neutral periodic box the split-BF16 M2L itself sits near 1e-4 in
    dV/dlambda (coarse-level multipoles are large and their operand rounding is coherent);
    the Hamiltonian form must not add to that: its errors equal the charge form's."""
    s = _systems()[1]
    eq = errors(run_gpu(s, precision="3xbf16"), oracle_ref(s, tol=1e-10))
    eh = errors(run_gpu(s, precision="3xbf16", interpolation="hamiltonian"), oracle_ref(s, hamiltonian=True, tol=1e-10))
    assert eh["F"] < 1e-4 and eh["E"] < 1e-4, eh
    assert eh["dVdl"] < 1.1 * eq["dVdl"] + 1e-6, (eh, eq)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_correction_alone_matches_oracle(which):
    s = _systems()[which]
    hc = oracle.hamiltonian_correction(s, tol=1e-11)
    gq = run_gpu(s, interpolation="charge")
    gh = run_gpu(s, interpolation="hamiltonian")
    dE = gh["E"] - gq["E"]
    assert dE == pytest.approx(hc["E"], rel=1e-5, abs=1e-6 * abs(gq["E"]))
    dV = gh["dVdl"] - gq["dVdl"]
    assert np.abs(dV - hc["dVdl"]).max() < 1e-5 * np.abs(hc["dVdl"]).max() + 1e-6 * np.abs(gq["dVdl"]).max()
    dF = gh["F"] - gq["F"]
    sites = s["site"] >= 0
    assert np.abs(dF[~sites]).max() == 0.0  # only site atoms change
    scale = np.abs(hc["F"]).max()
    assert np.abs(dF - hc["F"]).max() < 1e-4 * scale + 1e-6 * np.abs(gq["F"]).max()


def test_hamiltonian_energy_is_multilinear_on_gpu():
    """E_H(l1, l2) equals the bilinear interpolation of the charge-form energies at the
    corners, up to the FMM truncation error (itself quadratic in lambda, about 1e-5 of E
    here); the charge form misses that interpolation by far more."""
    s = synth.periodic_uniform(seed=33, n=2000, L=3.0, n_sites=2, site_size=5, neutral=False, p=10, depth=3)
    fq, d = make_solver(s, interpolation="charge")
    fh, _ = make_solver(s, interpolation="hamiltonian")

    def energy(f, lam):
        f.set_lambda(torch.tensor(lam, dtype=torch.float32, device="cuda"))
        E, _, dV, _ = f.eval(d["x"])
        torch.cuda.synchronize()
        return E.item(), dV.cpu().numpy().astype(np.float64)

    c = {(a, b): energy(fq, [a, b])[0] for a in (0.0, 1.0) for b in (0.0, 1.0)}
    l1, l2 = 0.375, 0.8125
    Eh, dVh = energy(fh, [l1, l2])
    bil = (1 - l1) * (1 - l2) * c[0, 0] + l1 * (1 - l2) * c[1, 0] + (1 - l1) * l2 * c[0, 1] + l1 * l2 * c[1, 1]
    scale = max(abs(v) for v in c.values())
    assert Eh == pytest.approx(bil, abs=4e-5 * scale)
    Eq, _ = energy(fq, [l1, l2])
    assert abs(Eq - bil) > 20 * abs(Eh - bil), (Eq - bil, Eh - bil)
    d1 = (1 - l2) * (c[1, 0] - c[0, 0]) + l2 * (c[1, 1] - c[0, 1])
    assert dVh[0] == pytest.approx(d1, rel=1e-3, abs=4e-5 * scale)
    fq.close()
    fh.close()


def test_hamiltonian_autograd_charge_gradients():
    """dE/dqB_i = k phi_i lambda + k lambda (1 - lambda) phi_h_i for site atoms (and minus the
    second term for qA), against the oracle."""
    s = _systems()[1]
    ref = oracle_ref(s, hamiltonian=True, tol=1e-10)
    d = to_dev(s)
    f, _ = make_solver(s, interpolation="hamiltonian")
    qA = d["qA"].clone().requires_grad_(True)
    qB = d["qB"].clone().requires_grad_(True)
    E = fmm_energy(d["x"], qA, qB, d["site"], d["lam"], f)
    E.backward()
    site = s["site"]
    lam_i = np.where(site >= 0, s["lam"][np.maximum(site, 0)], 0.0).astype(np.float64)
    w = lam_i * (1 - lam_i)
    gB = ref["phi"] * lam_i + oracle.KE_DEFAULT * w * ref["phi_h"]
    gA = ref["phi"] * (1 - lam_i) - oracle.KE_DEFAULT * w * ref["phi_h"]
    scale = np.abs(ref["phi"]).max()
    assert np.abs(qB.grad.double().cpu().numpy() - gB).max() < 1e-3 * scale
    assert np.abs(qA.grad.double().cpu().numpy() - gA).max() < 1e-3 * scale
    f.close()


def test_hamiltonian_mode_is_deterministic():
    s = _systems()[1]
    f, d = make_solver(s, interpolation="hamiltonian", precision="3xbf16")
    a = f.eval(d["x"], phi=True)
    b = f.eval(d["x"], phi=True)
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    f.close()
