"""fmm_binning_noalloc: the binning step for callers that cannot allocate device memory.

Some host programs own all of the GPU's memory (their own pool, a fixed budget) or run
loops that must not call cudaMalloc, which may synchronise the device.  For them the library
offers the binning step of an evaluation (Morton keys, stable sort, leaf ranges) with its
sort scratch in a static device array inside the library.  These tests call that entry point
through the C ABI and check it bit for bit:
  * against the binning that fmm_eval computes with its own buffers (fmm_get_binning), on
    calls in a row with different sizes, depths and sort pass counts (the scratch keeps the
    previous call's contents, so no call may depend on them);
  * against the oracle's binning specification at every depth 0..7 (0 to 3 radix passes,
    both parities of the pass count), including an open box with atoms outside it, which
    the status word reports;
  * at the scratch's capacity, FMM_NOALLOC_MAX_ATOMS atoms at depth 7.
The file is collected last, so that a failure here stops a run only after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2410_01626_b300 import FMM, binding

pytestmark = pytest.mark.gpu
MAX_ATOMS = 524288  # FMM_NOALLOC_MAX_ATOMS
FMM_DEV_DOMAIN = 1


def _noalloc(x_np, origin, L, periodic, depth, with_status=True):
    lib = binding.load()
    dev = torch.device("cuda")
    n = len(x_np)
    x = torch.from_numpy(np.ascontiguousarray(x_np, np.float32)).to(dev)
    key = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    nleaf = 1 << (3 * depth)
    start = torch.empty(nleaf, dtype=torch.int32, device=dev)
    count = torch.empty(nleaf, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    box = binding.FmmBox((ctypes.c_double * 3)(*origin), L)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = lib.fmm_binning_noalloc(ctypes.byref(box), int(periodic), depth, n, p(x), p(key), p(perm), p(start),
                                 p(count), p(status) if with_status else None,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    u32 = lambda t: t.cpu().numpy().view(np.uint32)  # noqa: E731
    return u32(key), u32(perm), u32(start), u32(count), int(status.item())


def _with_eval(s, depth, p=4):
    """The binning of fmm_eval (the handle's own buffers), read back with fmm_get_binning."""
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in ("x", "qA", "qB", "site", "lam")}
    f = FMM(s["L"], s["periodic"], p, depth, origin=s["origin"])
    f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
    f.eval(t["x"])
    out = [o.cpu().numpy().view(np.uint32) for o in f.binning()]
    torch.cuda.synchronize()
    f.close()
    return out


def _check_vs_oracle(x, origin, L, periodic, depth):
    got = _noalloc(x, origin, L, periodic, depth)
    ref = oracle.binning(x, origin, L, depth, periodic)
    for name, g, r in zip(("key", "perm", "start", "count"), got[:4], ref[:4]):
        assert np.array_equal(g, r), (name, depth, periodic)
    assert (got[4] & FMM_DEV_DOMAIN != 0) == (ref[4] != 0), (got[4], ref[4])
    return got[4]


@pytest.mark.parametrize("depth", range(8))
def test_noalloc_matches_the_oracle_binning_at_every_depth(depth):
    """Two calls in a row per depth: a periodic box with atoms wrapped from outside it, then an
    open box with a few atoms outside (status set) -- against the oracle's specification."""
    rng = np.random.default_rng(100 + depth)
    L, origin = 3.0, (0.25, -0.5, 1.0)
    x = np.asarray(origin) + rng.uniform(0.0, L, (5003, 3))
    x[:40] += rng.integers(-2, 3, (40, 3)) * L  # periodic images of the box
    assert _check_vs_oracle(x.astype(np.float32), origin, L, True, depth) == 0
    y = np.asarray(origin) + rng.uniform(0.0, L, (4097, 3))
    y[:3] = np.asarray(origin) + [L * 1.01, L / 2, L / 2]  # outside the open box: clamped, reported
    y[3] = np.asarray(origin) + L  # on the far faces: inside
    assert _check_vs_oracle(y.astype(np.float32), origin, L, False, depth) & FMM_DEV_DOMAIN


def test_noalloc_matches_eval_on_calls_in_a_row():
    """Against fmm_eval's own binning, calls in a row with different sizes and pass counts
    (depth 5: 2 passes, 1: 1 pass, 0: none, 3: 2 passes), the status pointer given or not."""
    cases = [(synth.periodic_uniform(seed=11, n=70000, L=4.0, p=4, depth=5), 5),
             (synth.open_uniform(seed=12, n=3001, L=3.0, n_sites=2, site_size=4), 1),
             (synth.periodic_uniform(seed=13, n=777, L=2.0, p=4, depth=0), 0),
             (synth.open_uniform(seed=14, n=20011, L=3.0, n_sites=2, site_size=4), 3)]
    for i, (s, depth) in enumerate(cases):
        got = _noalloc(s["x"], s["origin"], s["L"], s["periodic"], depth, with_status=i % 2 == 0)
        ref = _with_eval(s, depth)
        for g, r in zip(got[:4], ref):
            assert np.array_equal(g, r), depth
        assert got[4] == 0


def test_noalloc_at_capacity_depth_7():
    """FMM_NOALLOC_MAX_ATOMS atoms at depth 7 (2,097,152 leaves, three radix passes), twice in
    a row, against the oracle and against fmm_eval's binning."""
    s = synth.periodic_uniform(seed=15, n=MAX_ATOMS, L=5.0, p=1, depth=7)
    ref = oracle.binning(s["x"], s["origin"], s["L"], 7, True)
    ev = _with_eval(s, 7, p=1)
    for _ in range(2):
        got = _noalloc(s["x"], s["origin"], s["L"], True, 7)
        for name, g, r, e in zip(("key", "perm", "start", "count"), got[:4], ref[:4], ev):
            assert np.array_equal(g, r), name
            assert np.array_equal(g, e), name
        assert got[4] == 0


def test_noalloc_rejects_more_atoms_than_its_scratch():
    lib = binding.load()
    box = binding.FmmBox((ctypes.c_double * 3)(0.0, 0.0, 0.0), 1.0)
    st = lib.fmm_binning_noalloc(ctypes.byref(box), 1, 3, MAX_ATOMS + 1, None, None, None, None, None, None, None)
    assert st == 1  # FMM_ERR_ARG, nothing launched
