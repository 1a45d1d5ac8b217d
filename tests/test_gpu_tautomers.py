"""Sites with two lambda coordinates over four charge forms (Sec. 2.1, Eq. 2) on the GPU.

q_i = (1 - lp)[(1 - lt) qA + lt qB] + lp[(1 - lt) qC + lt qD]; dV/dlambda has (lp, lt) per
site.  Checked against the FP64 oracle in the charge and Hamiltonian forms, against the
two-form path for sites without tautomers, through autograd, and by finite differences.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from fmm_check import errors, oracle_ref
from paper_2410_01626_b300 import FMM, fmm_energy4

pytestmark = pytest.mark.gpu


def _dev4(s):
    d = {k: torch.from_numpy(np.ascontiguousarray(s[k])).cuda() for k in ("x", "qA", "qB", "qC", "qD", "site", "lam")}
    return d


def _solver4(s, precision="fp32", interpolation="charge"):
    f = FMM(s["L"], s["periodic"], s["p"], s["depth"], origin=s["origin"], precision=precision,
            interpolation=interpolation)
    d = _dev4(s)
    f.set_charges4(d["qA"], d["qB"], d["qC"], d["qD"], d["site"], d["lam"])
    return f, d


def _run4(s, **kw):
    f, d = _solver4(s, **kw)
    E, F, dV, _ = f.eval(d["x"])
    torch.cuda.synchronize()
    st = f.status_word()
    f.close()
    return {"E": E.item(), "F": F.cpu().numpy().astype(np.float64), "dVdl": dV.cpu().numpy().astype(np.float64),
            "status": st}


def _systems():
    return [
        synth.tautomer_sites(synth.open_uniform(seed=41, n=3000, L=4.0, n_sites=12, site_size=5, p=10, depth=3),
                             seed=1, tautomer_fraction=0.75),
        synth.tautomer_sites(synth.periodic_uniform(seed=42, n=3000, L=3.0, n_sites=12, site_size=5, p=10, depth=3),
                             seed=2, tautomer_fraction=0.75),
        synth.tautomer_sites(synth.solvated_30k(p=10), seed=3, tautomer_fraction=0.5),
    ]


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("interpolation", ["charge", "hamiltonian"])
def test_four_form_parity_with_oracle(which, interpolation):
    s = _systems()[which]
    tg = None if which < 2 else np.arange(0, len(s["x"]), 97)
    ref = oracle_ref(s, targets=tg, hamiltonian=interpolation == "hamiltonian", tol=1e-10)
    g = _run4(s, precision="3xtf32" if which < 2 else "3xbf16", interpolation=interpolation)
    e = errors(g, ref, idx=ref["idx"] if tg is not None else None)
    assert g["status"] == 0
    assert e["F"] < 1e-4 and e["dVdl"] < 1e-4, e
    if "E" in e:
        assert e["E"] < 1e-4, e
    assert g["dVdl"].shape == (2 * len(s["lam"]) // 2,)


@pytest.mark.parametrize("interpolation", ["charge", "hamiltonian"])
def test_four_form_without_tautomers_is_the_two_form_site(interpolation):
    s2 = synth.periodic_uniform(seed=43, n=2500, L=3.0, n_sites=10, site_size=4, p=8, depth=3)
    s4 = synth.tautomer_sites(s2, seed=4, tautomer_fraction=0.0)
    t2 = dict(s2)
    t2["lam"] = np.ascontiguousarray(s4["lam"][0::2])
    f2 = FMM(t2["L"], True, t2["p"], t2["depth"], precision="3xtf32", interpolation=interpolation)
    d2 = {k: torch.from_numpy(np.ascontiguousarray(t2[k])).cuda() for k in ("x", "qA", "qB", "site", "lam")}
    f2.set_charges(d2["qA"], d2["qB"], d2["site"], d2["lam"])
    E2, F2, dV2, _ = f2.eval(d2["x"])
    a = _run4(s4, precision="3xtf32", interpolation=interpolation)
    assert a["E"] == pytest.approx(E2.item(), rel=2e-6)
    F2 = F2.cpu().numpy()
    assert np.abs(a["F"] - F2).max() < 2e-5 * np.abs(F2).max()
    dv2 = dV2.cpu().numpy()
    assert np.abs(a["dVdl"][0::2] - dv2).max() < 2e-5 * np.abs(dv2).max()
    assert np.abs(a["dVdl"][1::2]).max() < 1e-5 * np.abs(dv2).max()
    f2.close()


@pytest.mark.parametrize("interpolation", ["charge", "hamiltonian"])
def test_four_form_autograd_charge_gradients(interpolation):
    s = _systems()[1]
    ref = oracle_ref(s, hamiltonian=interpolation == "hamiltonian", tol=1e-10)
    f, d = _solver4(s, precision="3xtf32", interpolation=interpolation)
    qs = [d[k].clone().requires_grad_(True) for k in ("qA", "qB", "qC", "qD")]
    lam = d["lam"].clone().requires_grad_(True)
    E = fmm_energy4(d["x"], *qs, d["site"], lam, f)
    E.backward()
    site = s["site"]
    l2 = s["lam"].astype(np.float64).reshape(-1, 2)
    p = np.where(site >= 0, l2[np.maximum(site, 0), 0], 0.0)
    t = np.where(site >= 0, l2[np.maximum(site, 0), 1], 0.0)
    w = np.stack([(1 - p) * (1 - t), (1 - p) * t, p * (1 - t), p * t], 1)
    w[site < 0] = [1.0, 0.0, 0.0, 0.0]
    gh = ref["g_h"] if "g_h" in ref else np.zeros((len(site), 4))
    scale = np.abs(ref["phi"]).max()
    for X in range(4):
        want = w[:, X] * (ref["phi"] + oracle.KE_DEFAULT * gh[:, X])
        got = qs[X].grad.double().cpu().numpy()
        assert np.abs(got - want).max() < 1e-3 * scale, X
    np.testing.assert_allclose(lam.grad.double().cpu().numpy(), ref["dVdl"], rtol=1e-3,
                               atol=1e-4 * np.abs(ref["dVdl"]).max())
    f.close()


def test_four_form_lambda_finite_differences():
    """Charge form: E is quadratic in every coordinate, so central differences of the GPU
    energy match dV/dlambda up to the energy's FP32 rounding."""
    s = _systems()[1]
    f, d = _solver4(s, precision="3xtf32")
    E, _, dV, _ = f.eval(d["x"])
    dV = dV.cpu().numpy()
    lam0 = d["lam"].clone()
    h = 0.0625
    for j in (0, 1, 6, 7):
        lp, lm = lam0.clone(), lam0.clone()
        lp[j] += h
        lm[j] -= h
        f.set_lambda(lp)
        Ep = f.eval(d["x"])[0].item()
        f.set_lambda(lm)
        Em = f.eval(d["x"])[0].item()
        fd = (Ep - Em) / (2 * h)
        assert fd == pytest.approx(dV[j], rel=2e-3, abs=2e-6 * abs(E.item()) / h)
    f.close()
