"""The near field's two source paths: staged and streamed.

One warp per target leaf copies its 27 neighbour leaves' atoms into shared memory when they fit
(640 atoms, the common case) and otherwise streams them neighbour by neighbour, one target per
lane.  A dense ball in a periodic background makes the leaves around the ball take the streamed
path and the others the staged one (the host counts the neighbourhoods to show that both run);
an open box at depth 1 puts every atom in every leaf's neighbourhood.  Each case is checked
against the FP64 oracle: the direct sum where the far field is absent, the Ewald sum otherwise.
"""
import numpy as np
import pytest

import synth
from fmm_check import errors, oracle_ref, run_gpu

pytestmark = pytest.mark.gpu
STAGE_CAP = 640  # atoms one warp stages


def neighbourhood_sizes(s, depth):
    """Atoms in each leaf's 27 neighbour leaves (periodic images included), the own leaf's
    count rounded up to even as the kernel pads it."""
    nb = 1 << depth
    cell = np.floor((s["x"].astype(np.float64) - np.asarray(s["origin"])) / (s["L"] / nb)).astype(np.int64)
    cell = cell % nb if s["periodic"] else np.clip(cell, 0, nb - 1)
    grid = np.zeros((nb, nb, nb), np.int64)
    np.add.at(grid, (cell[:, 0], cell[:, 1], cell[:, 2]), 1)
    tot = np.zeros_like(grid)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                if s["periodic"]:
                    tot += np.roll(grid, (-dx, -dy, -dz), (0, 1, 2))
                else:
                    sh = np.zeros_like(grid)
                    src = grid[max(dx, 0):nb + min(dx, 0), max(dy, 0):nb + min(dy, 0), max(dz, 0):nb + min(dz, 0)]
                    sh[max(-dx, 0):nb + min(-dx, 0), max(-dy, 0):nb + min(-dy, 0), max(-dz, 0):nb + min(-dz, 0)] = src
                    tot += sh
    return (tot + (grid & 1)).ravel()


@pytest.mark.parametrize("n", [500, 3000])
def test_open_depth1_equals_direct_sum(n):
    """Depth 1 in an open box: every leaf's neighbourhood is the whole system, so the near field
    is everything.  500 atoms are staged, 3000 streamed."""
    s = synth.open_uniform(seed=40 + n, n=n, L=3.0, n_sites=4, p=2, depth=1)
    assert (neighbourhood_sizes(s, 1).max() > STAGE_CAP) == (n > STAGE_CAP)
    ref = oracle_ref(s)
    g = run_gpu(s, depth=1)
    e = errors(g, ref)
    assert e["E"] < 1e-5 and e["F"] < 1e-5 and e["dVdl"] < 1e-5, e
    np.testing.assert_allclose(g["phi"], ref["phi"], rtol=0, atol=1e-5 * np.abs(ref["phi"]).max())
    assert g["status"] == 0


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_periodic_dense_ball_staged_and_streamed(precision):
    """A dense ball in a periodic background at depth 3: the leaves around the ball stream their
    sources, the others stage them; E, F and dV/dlambda against the Ewald oracle at p = 10."""
    s = synth.periodic_dense_cluster(seed=41)
    sizes = neighbourhood_sizes(s, 3)
    assert (sizes > STAGE_CAP).any() and (sizes <= STAGE_CAP).any(), sizes
    ref = oracle_ref(s)
    g = run_gpu(s, precision=precision)
    e = errors(g, ref)
    assert e["E"] < 1e-5 and e["F"] < 1e-4 and e["dVdl"] < 1e-4, e
    assert g["status"] == 0
