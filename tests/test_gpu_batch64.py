"""The batched workload against the oracle: 64 independent replicas of uneven size (N
log-uniform in 5k..50k atoms at 100 atoms/nm^3, water plus one cluster, 5..40 sites of 5
atoms; seeds 100..163; periodic, p = 8), each at the depth and kernel tiles the autotuner picks
(the fastest depth whose force and dV/dlambda errors, estimated against an order p + 2
evaluation, are within 0.7 x 1e-4), evaluated together through one Batch (parallel branches of
one CUDA graph) in the mixed precision the batched benchmark runs (FP16 M2L with split low
degrees).

Every replica is compared with the FP64 Ewald oracle on 160 random atoms plus every site atom
(so dV/dlambda is complete): relative RMS force error and dV/dlambda within 1e-4.  The TF32 form
is reported beside it (its dV/dlambda error is above 1e-4; it is not the batched precision).
"""
import numpy as np
import pytest
import torch

import synth
from fmm_check import errors, oracle_ref, to_dev
from paper_2410_01626_b300 import FMM, Batch
from paper_2410_01626_b300.autotune import TILES, tune

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _batch(reps, precision, depths=None):
    solvers, xs, chosen = [], [], []
    for i, s in enumerate(reps):
        d = to_dev(s)
        if depths is None:
            cfg, _ = tune(s["L"], True, s["p"], precision, d["x"], d["qA"], d["qB"], d["site"], d["lam"], reps=2,
                          tiles=TILES)
        else:
            cfg = {"depth": depths[i], "m2l_rows": 0, "p2p_warps": 0}
        dep = cfg["depth"]
        f = FMM(s["L"], True, s["p"], dep, precision=precision, m2l_rows=cfg["m2l_rows"], p2p_warps=cfg["p2p_warps"])
        f.set_charges(d["qA"], d["qB"], d["site"], d["lam"])
        solvers.append(f)
        xs.append(d["x"])
        chosen.append(dep)
    outs = [f.outputs() for f in solvers]
    b = Batch(solvers)
    b.eval_into(xs, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    torch.cuda.synchronize()
    status = [f.status_word() for f in solvers]
    res = [{"E": float(o[0].item()), "F": o[1].double().cpu().numpy(), "dVdl": o[2].double().cpu().numpy()}
           for o in outs]
    b.close()
    for f in solvers:
        f.close()
    return res, chosen, status


def test_batch64_replicas_match_the_oracle():
    reps = synth.replicas(64, first_seed=100)
    assert len(reps) == 64
    got, depths, status = _batch(reps, "fp16")
    assert all(st == 0 for st in status)
    worst = {"F": 0.0, "dVdl": 0.0}
    rows = []
    for i, (s, g) in enumerate(zip(reps, got)):
        tg = np.random.default_rng(1000 + i).choice(len(s["x"]), 160, replace=False)
        ref = oracle_ref(s, targets=tg, tol=1e-9)
        e = errors(g, ref, idx=ref["idx"])
        rows.append((len(s["x"]), depths[i], e["F"], e["dVdl"]))
        for k in worst:
            worst[k] = max(worst[k], e[k])
    for r in rows:
        print("N %6d depth %d  F %.2e  dVdl %.2e" % r)
    print("worst", worst)
    assert worst["F"] < 1e-4 and worst["dVdl"] < 1e-4, worst
