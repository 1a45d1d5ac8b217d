"""Repeated evaluations with the same buffers are replayed from a CUDA graph the library captures
itself (fmm_eval, fmm_eval_host).  The replay must give exactly what the same kernels give when
launched one by one, and must see what changed in the buffers it reads (positions, lambda)."""
import numpy as np
import pytest
import torch

import synth
from paper_2410_01626_b300 import FMM, pinned_empty

pytestmark = pytest.mark.gpu


def _solver(s, precision="3xbf16"):
    f = FMM(s["L"], s["periodic"], s["p"], s["depth"], precision=precision)
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).cuda() for k in ("x", "qA", "qB", "site", "lam")}
    f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
    return f, t


def _eager(s, x, lam, precision="3xbf16"):
    """Reference: a fresh handle in profiling mode, which always launches kernel by kernel."""
    f, t = _solver(s, precision)
    f.set_lambda(lam)
    f.set_profiling(True)
    E, F, dV, _ = f.eval(x)
    torch.cuda.synchronize()
    out = (E.clone(), F.clone(), dV.clone())
    f.close()
    return out


@pytest.mark.parametrize("precision", ["3xbf16", "fp16", "fp32"])
def test_replayed_evaluations_equal_eager_launches(precision):
    s = synth.solvated_30k()
    f, t = _solver(s, precision)
    n, K = len(s["x"]), len(s["lam"])
    x = t["x"].clone()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), device="cuda")
    dV = torch.zeros(K, device="cuda")
    ref = _eager(s, x, t["lam"], precision)
    for _ in range(4):  # eager, then captured and replayed, then replayed
        E.zero_(), F.zero_(), dV.zero_()
        f.eval_into(x, E, F, dV)
        torch.cuda.synchronize()
        assert torch.equal(E, ref[0]) and torch.equal(F, ref[1]) and torch.equal(dV, ref[2])
    # positions moved in place and lambda refreshed in place: the replay reads both
    x.add_(0.013)
    lam2 = (0.9 * t["lam"] + 0.05).contiguous()
    f.set_lambda(lam2)
    f.eval_into(x, E, F, dV)
    torch.cuda.synchronize()
    ref2 = _eager(s, x, lam2, precision)
    assert torch.equal(E, ref2[0]) and torch.equal(F, ref2[1]) and torch.equal(dV, ref2[2])
    assert f.status_word() == 0
    f.close()


def test_host_buffer_evaluations_repeat_exactly():
    s = synth.solvated_30k()
    f, t = _solver(s)
    n, K = len(s["x"]), len(s["lam"])
    xh = pinned_empty((n, 3))
    xh.copy_(torch.from_numpy(np.ascontiguousarray(s["x"])))
    outs = []
    for _ in range(3):
        Eh, Fh, dVh = pinned_empty(1, torch.float64), pinned_empty((n, 3)), pinned_empty(K)
        f.eval_host(xh, Eh, Fh, dVh)
        outs.append((Eh.clone(), Fh.clone(), dVh.clone()))
    ref = _eager(s, t["x"], t["lam"])
    for o in outs:
        assert torch.equal(o[0], ref[0].cpu()) and torch.equal(o[1], ref[1].cpu()) and torch.equal(o[2], ref[2].cpu())
    f.close()


@pytest.mark.parametrize("periodic,depth,side", [(True, 4, True), (False, 4, True), (False, 2, False)])
def test_stage_times_cover_the_branches(periodic, depth, side):
    """Profiling mode reports every stage of an evaluation; the coarse levels' side branch (M2L of
    levels below the two finest, root, their L2L) appears exactly when the tree has such levels."""
    from paper_2410_01626_b300 import STAGES
    if periodic:
        s = synth.periodic_uniform(seed=21, n=20000, L=4.0, n_sites=8, site_size=4, p=10, depth=depth)
    else:
        s = synth.open_uniform(seed=21, n=20000, L=4.0, n_sites=8, site_size=4, p=10, depth=depth)
    f = FMM(s["L"], s["periodic"], s["p"], s["depth"], origin=s["origin"], precision="3xbf16")
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).cuda() for k in ("x", "qA", "qB", "site", "lam")}
    f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
    f.set_profiling(True)
    f.eval(t["x"])
    ms = f.stage_times()
    f.close()
    assert list(ms) == list(STAGES)
    assert all(v >= 0.0 for v in ms.values()), ms
    for k in ("binning", "p2m", "m2l", "outputs", "final", "p2p"):
        assert ms[k] > 0.0, (k, ms)
    assert (ms["m2l_coarse"] > 0.0) == side and (ms["root"] > 0.0) == periodic, ms
