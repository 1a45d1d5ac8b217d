"""fmm_binning_noalloc: binning for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- code that runs while a stream is being
captured into a CUDA graph, programs that hand the GPU a fixed memory budget or
their own allocator, real-time loops.  For them the library offers the binning
step (Morton keys, stable sort, leaf ranges) with its sort scratch in a static
device array inside the library.  This test calls that entry point through the
C ABI and checks it against the binning that fmm_eval computes with its own
buffers, bit for bit, on two calls in a row (the scratch keeps the previous
call's contents, so the second call must not depend on them).
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2410_01626_b300 import FMM, binding

pytestmark = pytest.mark.gpu


def _noalloc(s, depth):
    lib = binding.load()
    dev = torch.device("cuda")
    n = len(s["x"])
    x = torch.from_numpy(np.ascontiguousarray(s["x"])).to(dev)
    key = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    nleaf = 1 << (3 * depth)
    start = torch.empty(nleaf, dtype=torch.int32, device=dev)
    count = torch.empty(nleaf, dtype=torch.int32, device=dev)
    box = binding.FmmBox((ctypes.c_double * 3)(*s["origin"]), s["L"])
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib.fmm_binning_noalloc(ctypes.byref(box), int(s["periodic"]), depth, n, p(x), p(key), p(perm), p(start),
                                 p(count), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    return key, perm, start, count


def _with_eval(s, depth):
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in ("x", "qA", "qB", "site", "lam")}
    f = FMM(s["L"], s["periodic"], 4, depth, origin=s["origin"])
    f.set_charges(t["qA"], t["qB"], t["site"], t["lam"])
    f.eval(t["x"])
    out = f.binning()
    torch.cuda.synchronize()
    f.close()
    return out


def test_noalloc_binning_matches_eval_two_calls():
    a = synth.periodic_uniform(seed=11, n=70000, L=4.0, p=4, depth=5)
    b = synth.open_uniform(seed=12, n=3001, L=3.0, n_sites=2, site_size=4)
    for s, depth in ((a, 5), (b, 3)):  # two calls in a row, different sizes and sort passes
        got = _noalloc(s, depth)
        ref = _with_eval(s, depth)
        for g, r in zip(got, ref):
            assert torch.equal(g, r)


def test_noalloc_rejects_more_atoms_than_its_scratch():
    lib = binding.load()
    box = binding.FmmBox((ctypes.c_double * 3)(0.0, 0.0, 0.0), 1.0)
    n = 524288 + 1  # FMM_NOALLOC_MAX_ATOMS + 1
    st = lib.fmm_binning_noalloc(ctypes.byref(box), 1, 3, n, None, None, None, None, None, None)
    assert st == 1  # FMM_ERR_ARG, nothing launched
