"""Parity at the full benchmark size: the solvated periodic system of 500,000
atoms (17 nm cube, 160,000 waters and four 5,000-atom clusters, 200 sites;
p = 10, depth 5), in the launch configuration the benchmark times (FP16 M2L with
split low degrees; the second call with the same buffers captures a CUDA graph
and later calls replay it), and in the split-BF16 and FP32 forms.

The FP64 oracle cannot evaluate all 500,000 atoms in seconds, so it computes
Ewald potentials and forces one target at a time for 400 random atoms plus
every site atom (which makes dV/dlambda complete).  Bars: relative RMS force
error <= 1e-4 for the mixed form at this size and dV/dlambda within 1e-4
relative; the FP32 CUDA-core path meets the same bars.  E needs every atom, so
it is checked through properties that hold at any size: E = 1/2 sum_i q_i phi_i
with the returned phi (k_e times the potential), and agreement of the tensor-core
and FP32 paths.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from fmm_check import errors, oracle_ref, to_dev
from paper_2410_01626_b300 import FMM

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def system():
    s = synth.solvated_500k()
    assert s["x"].shape == (500_000, 3) and s["periodic"] and s["p"] == 10 and s["depth"] == 5
    sample = np.random.default_rng(7).choice(len(s["x"]), 400, replace=False)
    ref = oracle_ref(s, targets=sample, tol=1e-8)
    return s, ref


def _evals(s, precision, calls):
    """`calls` evaluations into the same output buffers through one handle: eager launches,
    then the capture of a CUDA graph, then replays."""
    f = FMM(s["L"], True, s["p"], s["depth"], origin=s["origin"], precision=precision)
    d = to_dev(s)
    f.set_charges(d["qA"], d["qB"], d["site"], d["lam"])
    n, K = d["x"].shape[0], d["lam"].numel()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), device="cuda")
    dV = torch.zeros(K, device="cuda")
    phi = torch.zeros(n, device="cuda")
    outs = []
    for _ in range(calls):
        for t in (E, F, dV, phi):
            t.zero_()
        f.eval_into(d["x"], E, F, dV, phi)
        torch.cuda.synchronize()
        outs.append({"E": float(E.item()), "F": F.cpu().numpy().astype(np.float64),
                     "dVdl": dV.cpu().numpy().astype(np.float64), "phi": phi.cpu().numpy().astype(np.float64)})
    st = f.status_word()
    f.close()
    return outs, st


@pytest.fixture(scope="module")
def runs(system):
    s, _ = system
    h, st_h = _evals(s, "fp16", 3)
    bf, st_bf = _evals(s, "3xbf16", 1)
    fp, st_fp = _evals(s, "fp32", 1)
    assert st_h == 0 and st_bf == 0 and st_fp == 0
    return {"fp16": h, "3xbf16": bf, "fp32": fp}


@pytest.mark.parametrize("precision", ["fp16", "3xbf16", "fp32"])
def test_full_size_sampled_atoms_vs_oracle(system, runs, precision):
    s, ref = system
    g = runs[precision][-1]
    idx = ref["idx"]
    assert len(idx) >= 400 + 200 * 5 - 5  # the sample plus every site atom (overlaps allowed)
    e = errors(g, {"F": ref["F"], "dVdl": ref["dVdl"]}, idx)
    assert e["F"] < 1e-4 and e["dVdl"] < 1e-4, e
    # per-site worst case, measured against the larger of |ref_k| and the rms over sites
    dv = np.abs(g["dVdl"] - ref["dVdl"]) / np.maximum(np.abs(ref["dVdl"]), np.sqrt(np.mean(ref["dVdl"] ** 2)))
    assert dv.max() < 1e-3, dv.max()
    # the potential of the sampled atoms, relative to the largest sampled potential
    phi_ref = ref["phi"]
    assert np.abs(g["phi"][idx] - phi_ref).max() < 1e-4 * np.abs(phi_ref).max()


def test_full_size_graph_replay_repeats_the_eager_evaluation(runs):
    eager, captured, replayed = runs["fp16"]
    for k in ("F", "dVdl", "phi"):
        np.testing.assert_array_equal(captured[k], eager[k])
        np.testing.assert_array_equal(replayed[k], eager[k])
    assert captured["E"] == eager["E"] and replayed["E"] == eager["E"]


def test_full_size_energy_properties(system, runs):
    s, _ = system
    q, _ = oracle.charges(s["qA"], s["qB"], s["site"], s["lam"])
    for prec in ("fp16", "3xbf16", "fp32"):
        g = runs[prec][-1]
        e_phi = 0.5 * float(np.dot(q, g["phi"]))  # phi carries k_e
        assert abs(g["E"] - e_phi) < 1e-6 * abs(g["E"]), (prec, g["E"], e_phi)
    Ef = runs["fp32"][0]["E"]
    for prec in ("fp16", "3xbf16"):
        Eb = runs[prec][-1]["E"]
        assert abs(Eb - Ef) < 1e-5 * abs(Ef), (prec, Eb, Ef)
