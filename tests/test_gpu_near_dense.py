"""The near field's source paths.

One warp per target leaf copies its 27 neighbour leaves' atoms into shared memory when they fit
(592 atoms, the common case).  A larger neighbourhood is staged in rounds (a neighbour leaf split
across rounds where it does not fit), and a leaf above 64 atoms is split into work items of 64
targets that stage the whole neighbourhood the same way.  A dense ball in a periodic background exercises every path (the host counts
the leaves to show that each runs); an open box at depth 1 puts every atom in every leaf's
neighbourhood.  Each case is checked against the FP64 oracle: the direct sum where the far field
is absent, the Ewald sum otherwise.
"""
import numpy as np
import pytest

import synth
from fmm_check import errors, oracle_ref, run_gpu

pytestmark = pytest.mark.gpu
STAGE_CAP = 592  # atoms one warp stages
TILE = 64        # targets of one work item of a large leaf


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


def leaf_paths(s, depth):
    """Which near-field path each non-empty leaf takes: 'staged' (one piece), 'rounds' (a leaf of
    at most TILE atoms whose neighbourhood is staged in rounds) or 'items' (a leaf above TILE
    atoms, split into work items)."""
    nb = 1 << depth
    cell = np.floor((s["x"].astype(np.float64) - np.asarray(s["origin"])) / (s["L"] / nb)).astype(np.int64)
    cell = cell % nb if s["periodic"] else np.clip(cell, 0, nb - 1)
    grid = np.zeros((nb, nb, nb), np.int64).ravel()
    np.add.at(grid, np.ravel_multi_index((cell[:, 0], cell[:, 1], cell[:, 2]), (nb, nb, nb)), 1)
    total = neighbourhood_sizes(s, depth)
    paths = []
    for own, tot in zip(grid, total):
        if own == 0:
            continue
        if own > TILE:
            paths.append("items")
        else:
            paths.append("staged" if tot + (tot & 1) <= STAGE_CAP else "rounds")
    return paths


@pytest.mark.parametrize("n", [500, 3000])
def test_open_depth1_equals_direct_sum(n):
    """Depth 1 in an open box: every leaf's neighbourhood is the whole system, so the near field
    is everything.  At 500 atoms the leaves of at most 64 atoms are staged in one piece and the
    others are work items in one round; 3000 make every leaf a set of work items in rounds."""
    s = synth.open_uniform(seed=40 + n, n=n, L=3.0, n_sites=4, p=2, depth=1)
    paths = set(leaf_paths(s, 1))
    assert paths == ({"staged", "items"} if n < STAGE_CAP else {"items"}), paths
    ref = oracle_ref(s)
    g = run_gpu(s, depth=1)
    e = errors(g, ref)
    assert e["E"] < 1e-5 and e["F"] < 1e-5 and e["dVdl"] < 1e-5, e
    np.testing.assert_allclose(g["phi"], ref["phi"], rtol=0, atol=1e-5 * np.abs(ref["phi"]).max())
    assert g["status"] == 0


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_periodic_dense_ball_every_path(precision):
    """A dense ball in a periodic background at depth 3: the ball's leaves are large (work items),
    their neighbours stage in rounds, the others stage in one piece; E, F and dV/dlambda
    against the Ewald oracle at p = 10."""
    s = synth.periodic_dense_cluster(seed=41)
    paths = leaf_paths(s, 3)
    assert {"staged", "rounds", "items"} <= set(paths), sorted(set(paths))
    ref = oracle_ref(s)
    g = run_gpu(s, precision=precision)
    e = errors(g, ref)
    assert e["E"] < 1e-5 and e["F"] < 1e-4 and e["dVdl"] < 1e-4, e
    assert g["status"] == 0
