"""Failure paths, made on the host or by a wait that runs out -- never by a GPU fault.

* Bounded device waits: the tensor-core M2L is a pipeline of warps (bulk-copy producer, MMA
  issuer, accumulator drains) that wait on one another through shared-memory barriers; the
  tensor-core M2M and L2L wait for their operator copies and MMAs, and the near field for its
  staged atoms.  With the handle's wait limit set to one clock cycle, waits expire: the CTAs
  stop, drain what they issued and return; the evaluation reports FMM_DEV_TIMEOUT in the status
  word.  With the default limit restored, the same handle evaluates correctly again (eager,
  captured, replayed).
* Lost copies: the M2M/L2L and near-field waits are for bulk copies that land within the first
  poll, so a short limit alone does not make them expire.  fmm_inject_copy_loss makes those
  kernels announce their copies on the barriers without issuing them: the waits run out, the
  kernels stop and free what they hold, FMM_DEV_TIMEOUT is reported, and the handle recovers.
* Allocation failure: fmm_inject_alloc_failure makes the n-th device allocation of the library
  fail as if out of memory.  Creating a handle and setting its charges then returns FMM_ERR_OOM
  for every n up to the number of allocations they make, releases what they had allocated, and
  a handle made afterwards works.
"""
import numpy as np
import pytest
import torch

import synth
from fmm_check import errors, make_solver, oracle_ref, to_dev
from paper_2410_01626_b300 import FMM, FmmError, binding

pytestmark = pytest.mark.gpu
FMM_DEV_TIMEOUT = 4
FMM_ERR_OOM = 4


@pytest.mark.parametrize("precision", ["fp16", "3xbf16"])
def test_wait_limit_expires_then_the_handle_recovers(precision):
    s = synth.periodic_uniform(seed=3, n=3000, L=3.0, n_sites=8, site_size=4, p=10, depth=3)
    ref = oracle_ref(s)
    f, d = make_solver(s, precision=precision)
    f.set_wait_limit(1)
    f.eval(d["x"])
    torch.cuda.synchronize()
    assert f.status_word() & FMM_DEV_TIMEOUT
    f.set_wait_limit(0)  # the default, about 2 s
    for _ in range(3):  # eager launches, then graph capture, then a replay
        E, F, dV, phi = f.eval(d["x"], phi=True)
        torch.cuda.synchronize()
        g = {"E": float(E.item()), "F": F.double().cpu().numpy(), "dVdl": dV.double().cpu().numpy()}
        assert f.status_word() == 0
        e = errors(g, ref)
        assert e["F"] < 1e-4 and e["E"] < 1e-4 and e["dVdl"] < 1e-4, e
    f.close()


@pytest.mark.parametrize("mask,precision", [(1, "fp16"), (2, "fp32"), (3, "3xbf16")])
def test_lost_copies_time_out_then_the_handle_recovers(mask, precision):
    """mask 1: the tensor-core M2M/L2L operator copies (the tensor-core forms; FP32 mode
    translates on CUDA cores); 2: near-field staging; 3: both."""
    s = synth.periodic_uniform(seed=4, n=3000, L=3.0, n_sites=8, site_size=4, p=10, depth=3)
    ref = oracle_ref(s)
    f, d = make_solver(s, precision=precision)
    f.set_wait_limit(200000)  # about 0.1 ms: every lost copy's wait gives up quickly
    f.inject_copy_loss(mask)
    f.eval(d["x"])
    torch.cuda.synchronize()
    assert f.status_word() & FMM_DEV_TIMEOUT
    f.inject_copy_loss(0)
    f.set_wait_limit(0)
    for _ in range(3):  # eager launches, then graph capture, then a replay
        E, F, dV, phi = f.eval(d["x"], phi=True)
        torch.cuda.synchronize()
        g = {"E": float(E.item()), "F": F.double().cpu().numpy(), "dVdl": dV.double().cpu().numpy()}
        assert f.status_word() == 0
        e = errors(g, ref)
        assert e["F"] < 1e-4 and e["E"] < 1e-4 and e["dVdl"] < 1e-4, e
    with pytest.raises(FmmError):
        f.inject_copy_loss(4)
    f.close()


def _failure_sweep(lib, s, d):
    """Creation and set_charges with the k-th allocation failing, k = 1, 2, ... until one
    succeeds; returns the number of failures (each must be FMM_ERR_OOM)."""
    failures = 0
    try:
        for k in range(1, 64):
            assert lib.fmm_inject_alloc_failure(k) == 0
            try:
                f = FMM(s["L"], True, s["p"], s["depth"], precision="fp16")
                try:
                    f.set_charges(d["qA"], d["qB"], d["site"], d["lam"])
                finally:
                    f.close()
            except FmmError as exc:
                assert exc.code == FMM_ERR_OOM, exc
                failures += 1
                continue
            break  # k is past the last allocation: everything succeeded
    finally:
        lib.fmm_inject_alloc_failure(0)
    torch.cuda.synchronize()
    return failures


def test_allocation_failure_returns_oom_and_releases_memory():
    """The sweep runs twice: the first pass may leave what the driver reserves once per process
    (the same amount however often the calls run); the second must not lose device memory."""
    lib = binding.load()
    s = synth.periodic_uniform(seed=4, n=2000, L=3.0, n_sites=4, site_size=4, p=8, depth=3)
    d = to_dev(s)
    assert _failure_sweep(lib, s, d) >= 5  # operators, tensor-core banks, tree and atom buffers
    free0 = torch.cuda.mem_get_info()[0]
    assert _failure_sweep(lib, s, d) >= 5
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 16 << 20, (free0, free1)  # nothing of the failed calls is kept
    f, d2 = make_solver(s, precision="fp16")
    E, F, dV, _ = f.eval(d2["x"])
    torch.cuda.synchronize()
    g = {"E": float(E.item()), "F": F.double().cpu().numpy(), "dVdl": dV.double().cpu().numpy()}
    e = errors(g, oracle_ref(s))
    assert f.status_word() == 0 and e["F"] < 2e-4 and e["dVdl"] < 1e-4, e
    f.close()
    assert lib.fmm_inject_alloc_failure(-1) == 1  # FMM_ERR_ARG
