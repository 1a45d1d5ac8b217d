"""Trees of 6 and 7 levels, the deepest the library accepts (2,097,152 leaves at depth 7).

The tensor-core M2L covers trees of at most 5 levels, so the mixed precisions refuse deeper trees
(FMM_ERR_ARG, no silent change of precision); FP32 mode takes them, with the register-blocked
FP32 M2L. The test system is a sparse periodic one (20,000 atoms in a 4 nm cube), so most leaves
are empty. It runs at p = 8 in FP32 mode. Each run is checked against the FP64 Ewald oracle on 300
sampled atoms plus every site atom (which completes dV/dlambda), at the bars of p = 8 (relative
RMS force 2e-4, dV/dlambda 1e-4). The potentials give E = 1/2 sum q_i phi_i. Replays of the
captured graph equal the eager call bit for bit.
"""
import numpy as np
import pytest
import torch

import synth
from fmm_check import errors, make_solver, oracle_ref
from paper_2410_01626_b300 import FmmError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def system():
    s = synth.periodic_uniform(seed=70, n=20000, L=4.0, n_sites=8, site_size=4, p=8, depth=6)
    sample = np.random.default_rng(71).choice(len(s["x"]), 300, replace=False)
    return s, oracle_ref(s, targets=sample, tol=1e-9)


@pytest.mark.parametrize("depth", [6, 7])
def test_deep_tree_vs_oracle(system, depth):
    s, ref = system
    f, d = make_solver(s, depth=depth, precision="fp32")
    outs = []
    for _ in range(3):  # eager launches, then the graph's capture, then a replay
        E, F, dV, phi = f.eval(d["x"], phi=True)
        torch.cuda.synchronize()
        outs.append((float(E.item()), F.cpu().numpy(), dV.cpu().numpy(), phi.cpu().numpy()))
    assert f.status_word() == 0
    f.close()
    E0, F0, dV0, phi0 = outs[0]
    for Er, Fr, dVr, phir in outs[1:]:
        assert Er == E0 and np.array_equal(Fr, F0) and np.array_equal(dVr, dV0) and np.array_equal(phir, phi0)
    g = {"F": F0.astype(np.float64), "dVdl": dV0.astype(np.float64)}
    e = errors(g, {"F": ref["F"], "dVdl": ref["dVdl"]}, ref["idx"])
    assert e["F"] < 2e-4 and e["dVdl"] < 1e-4, e
    q = s["qA"].astype(np.float64) + np.where(s["site"] >= 0, s["lam"][np.maximum(s["site"], 0)], 0.0) * (
        s["qB"].astype(np.float64) - s["qA"].astype(np.float64))
    assert abs(E0 - 0.5 * float(np.dot(q, phi0.astype(np.float64)))) < 1e-4 * abs(E0), (E0,)


@pytest.mark.parametrize("precision", ["fp16", "3xbf16", "tf32"])
def test_mixed_precision_refuses_deep_trees(system, precision):
    s, _ = system
    for depth in (6, 7):
        with pytest.raises(FmmError) as exc:
            make_solver(s, depth=depth, precision=precision)
        assert exc.value.code == 1  # FMM_ERR_ARG
    f, _ = make_solver(s, depth=5, precision=precision)  # the deepest tree the tensor-core M2L takes
    f.close()
