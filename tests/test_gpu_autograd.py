"""Reverse-mode differentiation through the FMM energy (hand-written adjoint).

E(x, qA, qB, lambda) -> backward gives dE/dx = -F, dE/dqA, dE/dqB and
dE/dlambda = dV/dlambda.  Checked against the FP64 oracle's gradient and by
central finite differences of the GPU energy (E accumulated in FP64); the
differenced atoms are chosen away from leaf faces so the FMM approximation
does not switch leaves between the two evaluations.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from fmm_check import oracle_ref, to_dev
from paper_2410_01626_b300 import FMM, fmm_energy

pytestmark = pytest.mark.gpu


def _system():
    # the 30k-atom periodic system at p = 10, depth 4
    s = synth.solvated_30k(p=10)
    return s


@pytest.fixture(scope="module")
def sys30k():
    s = _system()
    return s, oracle_ref(s, targets=np.arange(0, len(s["x"]), 61), tol=1e-9)


def test_backward_matches_oracle_gradient(sys30k):
    s, ref = sys30k
    d = to_dev(s)
    solver = FMM(s["L"], True, s["p"], s["depth"])
    x = d["x"].clone().requires_grad_(True)
    qA = d["qA"].clone().requires_grad_(True)
    qB = d["qB"].clone().requires_grad_(True)
    lam = d["lam"].clone().requires_grad_(True)
    E = fmm_energy(x, qA, qB, d["site"], lam, solver)
    E.backward()
    idx = ref["idx"]
    gx = x.grad.double().cpu().numpy()[idx]
    # dE/dx = -F
    err_x = np.sqrt(((gx + ref["F"]) ** 2).sum() / (ref["F"] ** 2).sum())
    err_l = np.linalg.norm(lam.grad.double().cpu().numpy() - ref["dVdl"]) / np.linalg.norm(ref["dVdl"])
    assert err_x < 2e-4 and err_l < 1e-4, (err_x, err_l)
    # dE/dqA_i = k phi_i (1 - lambda_s), dE/dqB_i = k phi_i lambda_s (phi_i = the oracle's k*phi)
    site = s["site"][idx]
    lam_i = np.where(site >= 0, s["lam"][np.maximum(site, 0)], 0.0)
    gA_ref = ref["phi"] * (1 - lam_i)
    gB_ref = ref["phi"] * lam_i
    gA = qA.grad.double().cpu().numpy()[idx]
    gB = qB.grad.double().cpu().numpy()[idx]
    scale = np.abs(ref["phi"]).max()
    assert np.abs(gA - gA_ref).max() < 1e-3 * scale
    assert np.abs(gB - gB_ref).max() < 1e-3 * scale
    solver.close()


def test_finite_differences_in_x_and_lambda(sys30k):
    s, _ = sys30k
    d = to_dev(s)
    solver = FMM(s["L"], True, s["p"], s["depth"])
    x0 = d["x"].clone()
    x = x0.clone().requires_grad_(True)
    lam = d["lam"].clone().requires_grad_(True)
    E = fmm_energy(x, d["qA"], d["qB"], d["site"], lam, solver)
    E.backward()
    gx, gl = x.grad.clone(), lam.grad.clone()

    def energy(xx, ll):
        with torch.no_grad():
            return fmm_energy(xx, d["qA"], d["qB"], d["site"], ll, solver).item()

    # atoms at least 2 h_fd from every leaf face
    hleaf = s["L"] / 2 ** s["depth"]
    u = np.mod(s["x"].astype(np.float64), s["L"]) / hleaf
    frac = u - np.floor(u)
    ok = np.all((frac > 0.2) & (frac < 0.8), axis=1)
    rng = np.random.default_rng(3)
    atoms = rng.choice(np.nonzero(ok)[0], 32, replace=False)
    # FP32 positions: E carries ~1e-3 kJ/mol of rounding noise from all atoms' potentials, so
    # the step is 5e-3 nm (still 0.1 leaf edges inside the atom's leaf); the effective step is
    # taken from the rounded coordinates
    h = 5e-3
    errs = []
    for i in atoms:
        for a in range(3):
            xp = x0.clone(); xp[i, a] += h
            xm = x0.clone(); xm[i, a] -= h
            h_eff = (xp[i, a].double() - xm[i, a].double()).item() / 2
            fd = (energy(xp, lam.detach()) - energy(xm, lam.detach())) / (2 * h_eff)
            errs.append((fd, gx[i, a].item()))
    fd, an = np.array(errs).T
    assert np.linalg.norm(fd - an) / np.linalg.norm(an) < 1e-2, np.linalg.norm(fd - an) / np.linalg.norm(an)
    # E is exactly quadratic in lambda: the central difference is exact up to rounding
    hl = 1e-2
    for k in range(len(s["lam"])):
        lp = lam.detach().clone(); lp[k] += hl
        lm = lam.detach().clone(); lm[k] -= hl
        fdl = (energy(x0, lp) - energy(x0, lm)) / (2 * hl)
        assert fdl == pytest.approx(gl[k].item(), rel=2e-3, abs=1e-3 * gl.abs().max().item())
    solver.close()


def test_cuda_graph_replay_is_bitwise_equal():
    s = synth.periodic_uniform(seed=4, n=20000, L=5.0, p=8, depth=4)
    d = to_dev(s)
    for prec in ("fp32", "3xtf32", "3xbf16", "fp16"):
        f = FMM(s["L"], True, s["p"], s["depth"], precision=prec)
        f.set_charges(d["qA"], d["qB"], d["site"], d["lam"])
        E, F, dV, _ = f.outputs()
        f.eval_into(d["x"], E, F, dV)  # warm-up outside the capture
        torch.cuda.synchronize()
        ref = (E.clone(), F.clone(), dV.clone())
        g = torch.cuda.CUDAGraph()
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g, stream=stream):
                f.eval_into(d["x"], E, F, dV)
        for _ in range(3):
            E.zero_(); F.zero_(); dV.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(E, ref[0]) and torch.equal(F, ref[1]) and torch.equal(dV, ref[2])
        f.close()
