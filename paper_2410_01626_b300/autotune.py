"""Autotuner: tree depth (leaf tile) and kernel tiles per system, by timing, with accuracy as a
constraint.

The depth fixes the leaf size, which sets the balance between the pairwise near field (atoms
per leaf squared) and the multipole work (boxes per level); it also sets the accuracy at a given
order p: the far field's share of the force grows with depth, and with it the truncation error.
For each system the tuner times full evaluations at the heuristic depth round(log8(N / 16)) and
its neighbours (and, where the library offers them, the M2L tile widths and near-field block
shapes), estimates the relative force and dV/dlambda errors of each depth against one
evaluation at order p + 2 on the shallowest candidate tree (about 20 times more accurate), and
keeps the fastest configuration whose estimates are within the tolerances (times a safety
factor); when none is, the most accurate one.  Timing runs on the current stream with CUDA
events.
"""
from __future__ import annotations

import math

import torch

from .binding import FMM

TC_MAX_P = 10  # the tensor-core M2L forms hold (p + 1)^2 <= 128 coefficients


def depth_candidates(n_atoms: int, periodic: bool, lo: int = 1, hi: int = 5):
    d0 = int(min(hi, max(2, round(math.log(max(n_atoms, 16) / 16.0, 8)))))
    lo = max(lo, 1 if periodic else 2)
    return sorted({max(lo, d0 - 1), d0, min(hi, d0 + 1)})


def time_eval(solver: FMM, x: torch.Tensor, reps: int = 3) -> float:
    E, F, dV, _ = solver.outputs(x.device)
    solver.eval_into(x, E, F, dV)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        solver.eval_into(x, E, F, dV)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _rel(a, b):
    den = torch.linalg.norm(b.double())
    return float(torch.linalg.norm(a.double() - b.double()) / den) if float(den) > 0 else 0.0


def select_within_tolerance(table, f_tol=1e-4, dv_tol=1e-4, safety=0.7):
    """The fastest entry of {key: {"ms", "err_F", "err_dVdl"}} whose errors are within safety x
    the tolerances; when none is, the entry with the smallest error relative to its tolerance."""
    ok = [k for k, v in table.items() if v["err_F"] <= safety * f_tol and v["err_dVdl"] <= safety * dv_tol]
    if ok:
        return min(ok, key=lambda k: table[k]["ms"])
    return min(table, key=lambda k: max(table[k]["err_F"] / f_tol, table[k]["err_dVdl"] / dv_tol))


def tune(edge, periodic, p, precision, x, qA, qB, site, lam, origin=(0.0, 0.0, 0.0), candidates=None,
         reps: int = 3, f_tol: float = 1e-4, dv_tol: float = 1e-4, safety: float = 0.7, tiles=None):
    """Returns (config, table) for one system (device tensors): config = {"depth", "m2l_rows",
    "p2p_warps"}; table = {(depth, m2l_rows, p2p_warps): {"ms", "err_F", "err_dVdl"}} (errors
    for the depth candidates).  `tiles`: the (m2l_rows, p2p_warps) pairs tried at the chosen
    depth (None: the library defaults only; 0 selects a default)."""
    cands = candidates or depth_candidates(x.shape[0], periodic)
    tiles = tiles or [(0, 0)]
    # reference: order p + 2 on the shallowest candidate tree (FP32 where the tensor-core forms
    # do not hold that many coefficients)
    p_ref = p + 2
    ref_prec = precision if p_ref <= TC_MAX_P else "fp32"
    ref = FMM(edge, periodic, p_ref, min(cands), origin=origin, precision=ref_prec)
    ref.set_charges(qA, qB, site, lam)
    _, F_ref, dV_ref, _ = ref.eval(x)
    torch.cuda.synchronize()
    ref.close()
    table = {}

    def measure(d, rows, warps, with_error):
        try:
            f = FMM(edge, periodic, p, d, origin=origin, precision=precision, m2l_rows=rows, p2p_warps=warps)
        except Exception:
            return  # not offered at this depth / tile
        f.set_charges(qA, qB, site, lam)
        row = {}
        if with_error:
            _, F, dV, _ = f.eval(x)
            torch.cuda.synchronize()
            row["err_F"] = _rel(F, F_ref)
            row["err_dVdl"] = _rel(dV, dV_ref) if dV.numel() else 0.0
        row["ms"] = time_eval(f, x, reps)
        f.close()
        table[(d, rows, warps)] = row

    # (1) the depth, with the default tiles: the fastest within the error tolerances
    for d in cands:
        measure(d, 0, 0, True)
    best = select_within_tolerance(table, f_tol, dv_tol, safety)
    # (2) the tiles at that depth, by timing alone (every tile gives the same results)
    for (rows, warps) in tiles:
        if (best[0], rows, warps) not in table:
            measure(best[0], rows, warps, False)
    d0 = best[0]
    best = min((k for k in table if k[0] == d0), key=lambda k: table[k]["ms"])
    return {"depth": best[0], "m2l_rows": best[1], "p2p_warps": best[2]}, table


def tune_depth(edge, periodic, p, precision, x, qA, qB, site, lam, origin=(0.0, 0.0, 0.0), candidates=None,
               reps: int = 3, **kw):
    """Returns (best_depth, {depth: ms}) -- the depth part of ``tune`` with the default tiles."""
    cfg, table = tune(edge, periodic, p, precision, x, qA, qB, site, lam, origin, candidates, reps, **kw)
    return cfg["depth"], {k[0]: v["ms"] for k, v in table.items() if k[1:] == (0, 0)}


# (m2l_rows, p2p_warps) tried by the batch tuner.  Only one-warp near-field blocks: each replica is
# timed alone, where 2- or 4-warp blocks can look as fast, but beside other work (the multipole
# chain, other replicas) they take about twice as long as one-warp blocks (measured at 500k
# atoms: 0.39-0.43 against 0.20 ms in the step), and a batch is such concurrent work.
TILES = [(0, 0), (128, 0), (160, 0), (256, 0)]
