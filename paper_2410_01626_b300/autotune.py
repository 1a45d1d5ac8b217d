"""Tree-depth (leaf tile) autotuner.

The depth fixes the leaf size, which sets the balance between the pairwise near
field (atoms per leaf squared) and the multipole work (boxes per level).  For
each system the tuner times full evaluations at the heuristic depth
round(log8(N / 16)) and its neighbours and keeps the fastest; the chosen depth
is then used for the system's handle (for example inside a Batch).  Timing runs
on the current stream with CUDA events.
"""
from __future__ import annotations

import math

import torch

from .binding import FMM


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


def tune_depth(edge, periodic, p, precision, x, qA, qB, site, lam, origin=(0.0, 0.0, 0.0), candidates=None,
               reps: int = 3):
    """Returns (best_depth, {depth: ms}) for one system (device tensors)."""
    cands = candidates or depth_candidates(x.shape[0], periodic)
    times = {}
    for d in cands:
        try:
            f = FMM(edge, periodic, p, d, origin=origin, precision=precision)
        except Exception:
            continue  # the mode is not offered at this depth
        f.set_charges(qA, qB, site, lam)
        times[d] = time_eval(f, x, reps)
        f.close()
    best = min(times, key=times.get)
    return best, times
