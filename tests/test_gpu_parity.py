"""GPU parity of the CUDA FMM path against the FP64 oracle (direct sum / Ewald).

Tolerances: binning is bit-exact.  Where the far field is absent (open box,
depth <= 1) the result is a plain FP32 pair sum and must agree to FP32
rounding (1e-5 relative: a sum of ~1e3 terms of unit roundoff 6e-8 with
cancellation).  With the far field the multipole truncation dominates; the
bars are the ones stated for the method: relative RMS force error <= 1e-3 at
p = 6 and <= 1e-5 at p = 12, dV/dlambda within 1e-4 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from fmm_check import errors, make_solver, oracle_ref, run_gpu, to_dev

pytestmark = pytest.mark.gpu


# ---------------------------------------------------------------- binning (bit exact)
def _binning_case(s, depth):
    f, d = make_solver(s, depth=depth)
    E, F, dV, _ = f.eval(d["x"])
    key, perm, start, count = [t.cpu().numpy().view(np.uint32) for t in f.binning()]
    f.close()
    rk, rp, rs, rc, _ = oracle.binning(s["x"], s["origin"], s["L"], depth, s["periodic"])
    np.testing.assert_array_equal(key, rk)
    np.testing.assert_array_equal(perm, rp)
    np.testing.assert_array_equal(start, rs)
    np.testing.assert_array_equal(count, rc)


@pytest.mark.parametrize("depth", [0, 1, 2, 3, 5])
def test_binning_bit_exact_open(depth):
    _binning_case(synth.small_open(), depth)


@pytest.mark.parametrize("depth", [1, 4])
def test_binning_bit_exact_periodic_adversarial(depth):
    s = synth.periodic_uniform(seed=2, n=3000, L=2.0)
    x = s["x"].copy()
    L = s["L"]
    x[0] = [0, 0, 0]
    x[1] = [L, L, L]
    x[2] = [L / 2, L / 4, 3 * L / 8]
    x[3] = [-1e-7, -3 * L, 7.3 * L]
    x[4] = [2 * L, -L, 1.5 * L]
    x[5] = [-0.5 * L, 10.25 * L, -4.125 * L]
    s["x"] = x.astype(np.float32)
    _binning_case(s, depth)


@pytest.mark.parametrize("periodic", [True, False])
def test_binning_bit_exact_cell_faces(periodic):
    """Coordinates on cell faces and one or two float ulps either side of them, with a
    non-zero origin: the cases where single-precision key arithmetic would disagree with
    the FP64 specification."""
    depth, L, o = 4, 3.7, (-1.25, 0.5, 2.0)
    s = synth.open_uniform(seed=9, n=4000, L=L, n_sites=2)
    s["origin"] = o
    h = L / 2 ** depth
    rng = np.random.default_rng(4)
    x = (s["x"].astype(np.float64) + np.asarray(o)).astype(np.float32)
    k = rng.integers(0, 2 ** depth + 1, size=(3000, 3))
    face = (np.asarray(o) + k * h).astype(np.float32)
    ulps = rng.integers(-2, 3, size=face.shape)
    face = np.nextafter(face, np.where(ulps > 0, np.inf, -np.inf).astype(np.float32))
    face = np.where(ulps == 0, (np.asarray(o) + k * h).astype(np.float32), face)
    x[:3000] = face
    if not periodic:  # keep the open box's atoms inside [origin, origin + L]
        x = np.clip(x, np.asarray(o, np.float32), np.asarray(o) + L).astype(np.float32)
    s["x"] = x
    s["periodic"] = periodic
    _binning_case(s, depth)


def test_binning_large_stable():
    """Many atoms per leaf and ties: the permutation must be the stable one."""
    rng = np.random.default_rng(0)
    s = synth.open_uniform(seed=1, n=200000, L=4.0, n_sites=1)
    s["x"][: 100000] = np.round(s["x"][: 100000], 1)  # heavy duplication of positions
    _binning_case(s, 5)


@pytest.mark.parametrize("depth", [6, 7])
def test_binning_bit_exact_deep_trees(depth):
    """Deep trees: the leaf-count scan runs over many tiles (64 and 512 at depths 6 and 7),
    most leaves empty; low p keeps the rest of the evaluation cheap."""
    s = synth.open_uniform(seed=12, n=300000, L=4.0, n_sites=2, p=2, depth=depth)
    _binning_case(s, depth)


# ---------------------------------------------------------------- near field only
@pytest.mark.parametrize("depth", [0, 1])
def test_open_near_field_only_equals_direct_sum(depth):
    s = synth.small_open()
    ref = oracle_ref(s)
    g = run_gpu(s, depth=depth)
    e = errors(g, ref)
    assert e["E"] < 1e-5 and e["F"] < 1e-5 and e["dVdl"] < 1e-5, e
    np.testing.assert_allclose(g["phi"], ref["phi"], rtol=0, atol=1e-5 * np.abs(ref["phi"]).max())
    assert g["status"] == 0


# ---------------------------------------------------------------- degenerate inputs
@pytest.mark.parametrize("periodic", [True, False])
def test_empty_system(periodic):
    """No atoms and no sites: the evaluation runs (every tree stage over empty leaves) and gives
    E = 0 exactly, empty F, phi and dV/dlambda, and no device status."""
    from paper_2410_01626_b300 import FMM
    f = FMM(3.0, periodic, 8, 3, origin=(0.0, 0.0, 0.0))
    z = torch.zeros(0, device="cuda")
    f.set_charges(z, z.clone(), torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"))
    for _ in range(3):  # eager, graph capture, replay
        E, F, dV, phi = f.eval(torch.zeros((0, 3), device="cuda"), phi=True)
        torch.cuda.synchronize()
        assert float(E.item()) == 0.0
        assert tuple(F.shape) == (0, 3) and dV.numel() == 0 and phi.numel() == 0
    assert f.status_word() == 0
    f.close()


def test_no_sites():
    """Atoms without titratable sites (K = 0): E and F as the oracle's, no dV/dlambda."""
    s = dict(synth.small_open())
    s["site"] = np.full_like(s["site"], -1)
    s["lam"] = np.zeros(0, dtype=np.float32)
    s["qB"] = s["qA"].copy()
    ref = oracle_ref(s)
    g = run_gpu(s, p=10, depth=2)
    assert g["dVdl"].size == 0 and g["status"] == 0
    e = errors(g, ref)
    assert e["E"] < 1e-4 and e["F"] < 1e-4, e


# ---------------------------------------------------------------- open boundary FMM
@pytest.mark.parametrize("p,ftol", [(6, 1e-3), (8, 2e-4), (12, 1e-5)])
def test_open_fmm_small(p, ftol):
    s = synth.small_open()
    ref = oracle_ref(s)
    e = errors(run_gpu(s, p=p, depth=2), ref)
    assert e["F"] < ftol, e
    assert e["dVdl"] < 1e-4, e
    assert e["E"] < 1e-4, e


def test_open_fmm_depth3_ragged():
    """Several levels of far field, empty leaves, a ragged leaf population."""
    s = synth.open_uniform(seed=4, n=5003, L=6.0, n_sites=12, site_size=5)
    ref = oracle_ref(s)
    e = errors(run_gpu(s, p=10, depth=3), ref)
    assert e["F"] < 1e-4 and e["dVdl"] < 1e-4 and e["E"] < 1e-4, e


# ---------------------------------------------------------------- periodic FMM
@pytest.mark.parametrize("neutral", [True, False])
def test_periodic_fmm_small(neutral):
    s = synth.periodic_uniform(seed=3, n=2000, L=3.0, n_sites=8, site_size=4, neutral=neutral, p=8, depth=3)
    ref = oracle_ref(s)
    e = errors(run_gpu(s), ref)
    assert e["F"] < 2e-4 and e["dVdl"] < 1e-4 and e["E"] < 1e-4, e


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_periodic_shallow_trees(depth):
    s = synth.periodic_uniform(seed=8, n=300, L=1.7, n_sites=3, site_size=4, neutral=False, p=10, depth=depth)
    ref = oracle_ref(s)
    e = errors(run_gpu(s), ref)
    assert e["F"] < 1e-4 and e["dVdl"] < 1e-4 and e["E"] < 1e-4, e


@pytest.mark.parametrize("p,tol", [(8, 5e-5), (12, 5e-6)])
def test_periodic_single_charge_wigner(p, tol):
    """One charge and its images: E = k q^2 xi / (2L).  A wrong background or
    self-image convention is an O(1) error; what remains is FMM truncation."""
    s = synth.periodic_uniform(seed=0, n=1, L=2.0, n_sites=0, site_size=1, neutral=False, p=p, depth=2)
    s["qA"][:] = 1.0
    s["qB"][:] = 1.0
    g = run_gpu(s)
    E_ref = 0.5 * oracle.KE_DEFAULT * (-2.8372974794) / 2.0
    assert g["E"] == pytest.approx(E_ref, rel=tol)
    # the exact force vanishes by symmetry; compare with the natural scale k q^2 / L^2
    assert np.abs(g["F"]).max() < 20 * tol * oracle.KE_DEFAULT / 2.0 ** 2


def test_periodic_nacl_madelung():
    a = 0.5640
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    na = np.concatenate([base + [i, j, k] for i in range(4) for j in range(4) for k in range(4)]) * a
    # shifted by a/4 so that every ion sits at a leaf centre of the depth-3 tree (an ion on a
    # leaf corner is the worst case of the expansions; the lattice energy is shift invariant)
    x = (np.concatenate([na, na + [0.5 * a, 0, 0]]) + a / 4).astype(np.float32)
    q = np.concatenate([np.ones(len(na)), -np.ones(len(na))]).astype(np.float32)
    s = {"name": "nacl", "x": x, "qA": q, "qB": q.copy(), "site": np.full(len(q), -1, np.int32),
         "lam": np.zeros(0, np.float32), "L": 4 * a, "origin": (0.0, 0.0, 0.0), "periodic": True, "p": 10, "depth": 3}
    g = run_gpu(s)
    M = -g["E"] / oracle.KE_DEFAULT * (a / 2) / (len(q) / 2)
    assert M == pytest.approx(1.747565, abs=2e-5)


@pytest.mark.slow
def test_periodic_solvated_30k():
    s = synth.solvated_30k()
    ref = oracle_ref(s, tol=1e-9)
    g = run_gpu(s)
    e = errors(g, ref)
    assert e["F"] < 2e-4 and e["dVdl"] < 1e-4 and e["E"] < 1e-4, e
    assert g["status"] == 0


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_periodic_solvated_30k_charge_buffers(precision):
    """The 30k system with a charge buffer per site (Sec. 2.5): neutral at every lambda, so
    the background term vanishes and the periodic FMM alone must match Ewald, at the same
    bars as the non-neutral base system (where the background term carries the net charge)."""
    s = synth.solvated_30k_buf()
    ref = oracle_ref(s, tol=1e-9)
    g = run_gpu(s, precision=precision)
    e = errors(g, ref)
    assert e["F"] < 2e-4 and e["dVdl"] < 1e-4 and e["E"] < 1e-4, e
    assert g["status"] == 0


@pytest.mark.slow
def test_periodic_p12_force_accuracy():
    """p = 12 in a periodic box: the relative RMS force error against Ewald at most 1e-5
    (the p = 12 bar), on the 30k solvated system at depth 4 (1,000 sampled atoms plus the
    site atoms)."""
    s = synth.solvated_30k(p=12)
    tg = np.random.default_rng(12).choice(len(s["x"]), 1000, replace=False)
    ref = oracle_ref(s, targets=tg, tol=1e-10)
    g = run_gpu(s)
    e = errors(g, ref, idx=ref["idx"])
    print(f"periodic p=12: {e}")
    assert e["F"] < 1e-5 and e["dVdl"] < 1e-4, e
    assert g["status"] == 0


# ---------------------------------------------------------------- API behaviour
def test_deterministic_bitwise():
    s = synth.periodic_uniform(seed=3, n=4000, L=3.0, p=8, depth=3)
    f, d = make_solver(s)
    a = f.eval(d["x"], phi=True)
    b = f.eval(d["x"], phi=True)
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    f.close()


def test_eval_host_matches_device():
    s = synth.periodic_uniform(seed=6, n=3000, L=3.0, p=8, depth=3)
    f, d = make_solver(s)
    E, F, dV, _ = f.eval(d["x"])
    torch.cuda.synchronize()
    xh = torch.from_numpy(s["x"]).pin_memory()
    Eh = torch.empty(1, dtype=torch.float64).pin_memory()
    Fh = torch.empty(len(s["x"]), 3).pin_memory()
    dVh = torch.empty(len(s["lam"])).pin_memory()
    f.eval_host(xh, Eh, Fh, dVh)
    assert Eh.item() == E.item()
    assert torch.equal(Fh, F.cpu()) and torch.equal(dVh, dV.cpu())
    # the same through buffers from the library's page-locked allocator
    from paper_2410_01626_b300 import pinned_empty
    xp = pinned_empty(xh.shape)
    xp.copy_(xh)
    Ep, Fp, dVp = pinned_empty(1, torch.float64), pinned_empty(Fh.shape), pinned_empty(dVh.shape)
    f.eval_host(xp, Ep, Fp, dVp)
    assert Ep.item() == E.item()
    assert torch.equal(Fp, F.cpu()) and torch.equal(dVp, dV.cpu())
    del xp, Ep, Fp, dVp  # released through fmm_host_free
    f.close()


def test_eval_host_async_calls_in_flight_match_device():
    """Several fmm_eval_host_async calls in flight on one stream (different positions each, so
    consecutive calls use the two staging sets in turn and overlap a copy with the previous
    evaluation), then one synchronisation: every call's results equal fmm_eval's on the device
    with its positions, bit for bit -- also with a synchronous fmm_eval_host in between and once
    the staging sets' graphs are captured and replayed."""
    s = synth.periodic_uniform(seed=6, n=3000, L=3.0, p=8, depth=3)
    f, d = make_solver(s, precision="fp16")
    rng = np.random.default_rng(3)
    xs = [np.ascontiguousarray((s["x"] + rng.uniform(-0.01, 0.01, s["x"].shape)).astype(np.float32))
          for _ in range(6)]
    refs = []
    for x in xs:
        E, F, dV, _ = f.eval(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        refs.append((E.item(), F.cpu(), dV.cpu()))
    n, K = len(s["x"]), len(s["lam"])
    bufs = [(torch.from_numpy(x).pin_memory(), torch.empty(1, dtype=torch.float64).pin_memory(),
             torch.empty(n, 3).pin_memory(), torch.empty(K).pin_memory()) for x in xs]
    for rnd in range(3):  # eager, then capture of both staging sets' graphs, then replays
        for i, (xh, Eh, Fh, dVh) in enumerate(bufs):
            if rnd == 1 and i == 3:
                f.eval_host(xh, Eh, Fh, dVh)  # a synchronous call between asynchronous ones
            else:
                f.eval_host_async(xh, Eh, Fh, dVh)
        torch.cuda.synchronize()
        for (xh, Eh, Fh, dVh), (E, F, dV) in zip(bufs, refs):
            assert Eh.item() == E
            assert torch.equal(Fh, F) and torch.equal(dVh, dV)
            Eh.zero_(); Fh.zero_(); dVh.zero_()
    assert f.status_word() == 0
    f.close()


def test_evaluations_on_two_streams_in_turn_match_device():
    """fmm_eval_host_async and fmm_eval calls alternating between two streams, several in
    flight, with different positions each: the handle orders its evaluations across the
    streams (each waits for the previous evaluation's kernels, not for its result copies), so
    every call's results equal a one-at-a-time device evaluation bit for bit -- eager, captured
    and replayed.  fmm_stream_wait_eval orders a caller's own work (here an L2-sized write
    that the next evaluation must not overlap) after the previous evaluation."""
    s = synth.periodic_uniform(seed=6, n=3000, L=3.0, p=8, depth=3)
    f, d = make_solver(s, precision="fp16")
    rng = np.random.default_rng(4)
    xs = [np.ascontiguousarray((s["x"] + rng.uniform(-0.01, 0.01, s["x"].shape)).astype(np.float32))
          for _ in range(6)]
    refs = []
    for x in xs:
        E, F, dV, _ = f.eval(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        refs.append((E.item(), F.cpu(), dV.cpu()))
    n, K = len(s["x"]), len(s["lam"])
    bufs = [(torch.from_numpy(x).pin_memory(), torch.empty(1, dtype=torch.float64).pin_memory(),
             torch.empty(n, 3).pin_memory(), torch.empty(K).pin_memory()) for x in xs]
    dev = [(torch.from_numpy(x).cuda(), torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty(n, 3, device="cuda"), torch.empty(K, device="cuda")) for x in xs]
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    scratch = torch.empty(64 << 20, device="cuda")
    torch.cuda.synchronize()
    for rnd in range(3):  # eager, then capture of both staging sets' graphs, then replays
        for i, (xh, Eh, Fh, dVh) in enumerate(bufs):
            with torch.cuda.stream(streams[i & 1]):
                f.stream_wait_eval()
                scratch.zero_()
                f.eval_host_async(xh, Eh, Fh, dVh)
        torch.cuda.synchronize()
        for (xh, Eh, Fh, dVh), (E, F, dV) in zip(bufs, refs):
            assert Eh.item() == E
            assert torch.equal(Fh, F) and torch.equal(dVh, dV)
            Eh.zero_(); Fh.zero_(); dVh.zero_()
        for i, (x, E, F, dV) in enumerate(dev):  # device buffers, the same alternation
            with torch.cuda.stream(streams[i & 1]):
                f.eval_into(x, E, F, dV)
        torch.cuda.synchronize()
        for (x, E, F, dV), (Er, Fr, dVr) in zip(dev, refs):
            assert E.item() == Er
            assert torch.equal(F.cpu(), Fr) and torch.equal(dV.cpu(), dVr)
            F.zero_()
    assert f.status_word() == 0
    f.close()


def test_open_domain_error_is_reported():
    s = synth.small_open()
    s["x"][5] = [4.5, 1.0, 1.0]
    f, d = make_solver(s)
    f.eval(d["x"])
    assert f.status_word() & 1
    assert f.status_word() == 0  # cleared by the read
    f.close()


def test_set_lambda_changes_only_charges():
    s = synth.small_open()
    f, d = make_solver(s)
    lam2 = torch.rand_like(d["lam"])
    f.set_lambda(lam2)
    E, F, dV, _ = f.eval(d["x"])
    s2 = dict(s, lam=lam2.cpu().numpy())
    ref = oracle.evaluate(s2)
    e = errors({"E": E.item(), "F": F.cpu().numpy(), "dVdl": dV.cpu().numpy()}, ref)
    assert e["F"] < 2e-4 and e["dVdl"] < 1e-4, e
    f.close()


def test_bad_arguments_rejected_on_host():
    from paper_2410_01626_b300 import FMM, FmmError
    with pytest.raises(FmmError):
        FMM(-1.0, False, 8, 2)
    with pytest.raises(FmmError):
        FMM(1.0, False, 0, 2)
    with pytest.raises(FmmError):
        FMM(1.0, False, 8, 9)
    f = FMM(1.0, False, 4, 1)
    q = torch.zeros(3, device="cuda")
    with pytest.raises(FmmError):
        f.set_charges(q, q, torch.tensor([0, 5, -1], dtype=torch.int32, device="cuda"), torch.zeros(2, device="cuda"))
    with pytest.raises(FmmError):  # eval before charges
        f.eval_into(torch.zeros(0, 3, device="cuda"), torch.zeros(1, dtype=torch.float64, device="cuda"))
    f.close()


# ---------------------------------------------------------------- tensor-core M2L (TF32)
@pytest.mark.parametrize("periodic,p,depth", [(True, 8, 3), (True, 10, 3), (False, 8, 2), (False, 10, 4), (True, 10, 1)])
def test_tf32_m2l_parity(periodic, p, depth):
    """TF32 operands (rounded to nearest) with FP32 accumulation: forces stay within
    1e-4 of the oracle; the potential (E, dV/dlambda) carries the operand rounding
    (2^-11 relative per operand), measured at about 1e-3 and bounded here by 5e-3."""
    if periodic:
        s = synth.periodic_uniform(seed=3, n=3000, L=3.0, n_sites=8, site_size=4, p=p, depth=depth)
    else:
        s = synth.open_uniform(seed=5, n=3000, L=5.0, n_sites=8, site_size=4, p=p, depth=depth)
    ref = oracle_ref(s)
    g = run_gpu(s, precision="tf32")
    e = errors(g, ref)
    assert g["status"] == 0
    assert e["F"] < 1e-4 and e["E"] < 5e-3 and e["dVdl"] < 5e-3, e


def test_tf32_mode_unavailable_is_refused():
    from paper_2410_01626_b300 import FMM, FmmError
    with pytest.raises(FmmError):
        FMM(1.0, True, 12, 3, precision="tf32")  # 169 coefficients exceed one 128-row MMA


@pytest.mark.parametrize("periodic,p,depth", [(True, 8, 3), (True, 10, 3), (False, 10, 4), (True, 10, 1)])
def test_3xtf32_m2l_parity(periodic, p, depth):
    """Split TF32 (hi*hi + hi*lo + lo*hi) restores FP32-level operands: E, F and
    dV/dlambda all within 1e-4 of the oracle, like the FP32 path."""
    if periodic:
        s = synth.periodic_uniform(seed=3, n=3000, L=3.0, n_sites=8, site_size=4, p=p, depth=depth)
    else:
        s = synth.open_uniform(seed=5, n=3000, L=5.0, n_sites=8, site_size=4, p=p, depth=depth)
    ref = oracle_ref(s)
    g = run_gpu(s, precision="3xtf32")
    e = errors(g, ref)
    assert g["status"] == 0
    assert e["F"] < 1e-4 and e["E"] < 1e-4 and e["dVdl"] < 1e-4, e


# ---------------------------------------------------------------- tensor-core M2L (split BF16)
@pytest.mark.parametrize("periodic,p,depth", [(True, 8, 3), (True, 10, 3), (False, 8, 2), (False, 10, 4), (True, 10, 1)])
def test_3xbf16_m2l_parity(periodic, p, depth):
    """Split BF16 (hi*hi + hi*lo + lo*hi, about 16 significant bits per operand, products
    exact in FP32): E, F and dV/dlambda within 1e-4 of the oracle."""
    if periodic:
        s = synth.periodic_uniform(seed=3, n=3000, L=3.0, n_sites=8, site_size=4, p=p, depth=depth)
    else:
        s = synth.open_uniform(seed=5, n=3000, L=5.0, n_sites=8, site_size=4, p=p, depth=depth)
    ref = oracle_ref(s)
    g = run_gpu(s, precision="3xbf16")
    e = errors(g, ref)
    print(f"3xbf16 periodic={periodic} p={p} depth={depth}: {e}")
    assert g["status"] == 0
    assert e["F"] < 1e-4 and e["E"] < 1e-4 and e["dVdl"] < 1e-4, e


def test_3xbf16_close_to_fp32_path():
    """Each split BF16 operand carries up to 2^-16 relative error (hi and lo keep 8
    significant bits each) and the dropped lo*lo product is of the same order, so the
    local expansions differ from the FP32 path by about 1e-5 of the summed term sizes.
    Forces are near-field dominated (measured 2e-7); E and dV/dlambda sum potentials whose
    far-field terms cancel (measured 1.5e-6 and 4.5e-5).  A wrong cell layout or
    descriptor shows as an O(1) difference."""
    s = synth.periodic_uniform(seed=11, n=6000, L=3.5, n_sites=8, site_size=4, p=10, depth=3)
    a = run_gpu(s, precision="fp32")
    b = run_gpu(s, precision="3xbf16")
    dF = np.sqrt(((a["F"] - b["F"]) ** 2).sum() / (a["F"] ** 2).sum())
    dE = abs(a["E"] - b["E"]) / abs(a["E"])
    dV = np.linalg.norm(a["dVdl"] - b["dVdl"]) / np.linalg.norm(a["dVdl"])
    print(f"3xbf16 vs fp32: dF {dF:.2e} dE {dE:.2e} dVdl {dV:.2e}")
    assert dF < 2e-6 and dE < 1e-5 and dV < 1e-4, (dF, dE, dV)


# ---------------------------------------------------------------- tensor-core M2L (FP16, split low degrees)
@pytest.mark.parametrize("periodic,p,depth", [(True, 8, 3), (True, 10, 3), (False, 8, 2), (False, 10, 4), (True, 10, 1)])
def test_fp16_m2l_parity(periodic, p, depth):
    """FP16 M2L: the input coefficients of degrees 0..3 as split hi/lo operands (three
    products, about 22 bits), every higher degree as one FP16 product (11 bits).  E, F and
    dV/dlambda within 1e-4 of the oracle, like the FP32 path."""
    if periodic:
        s = synth.periodic_uniform(seed=3, n=3000, L=3.0, n_sites=8, site_size=4, p=p, depth=depth)
    else:
        s = synth.open_uniform(seed=5, n=3000, L=5.0, n_sites=8, site_size=4, p=p, depth=depth)
    ref = oracle_ref(s)
    g = run_gpu(s, precision="fp16")
    e = errors(g, ref)
    print(f"fp16 periodic={periodic} p={p} depth={depth}: {e}")
    assert g["status"] == 0
    assert e["F"] < 1e-4 and e["E"] < 1e-4 and e["dVdl"] < 1e-4, e


@pytest.mark.parametrize("periodic,p,depth", [(True, 4, 3), (True, 5, 3), (False, 6, 3), (True, 6, 3)])
def test_fp16_m2l_low_orders_add_nothing_to_truncation(periodic, p, depth):
    """At p = 4..6 the expansion's truncation error (1e-3 and above) dominates: the FP16 form
    must add nothing to it -- its errors against the oracle equal the FP32 path's.  These
    orders cover the other shapes of the K chunks (ncp = 32, 48, 64: a last chunk of one or
    two K steps)."""
    if periodic:
        s = synth.periodic_uniform(seed=3, n=3000, L=3.0, n_sites=8, site_size=4, p=p, depth=depth)
    else:
        s = synth.open_uniform(seed=5, n=3000, L=5.0, n_sites=8, site_size=4, p=p, depth=depth)
    ref = oracle_ref(s)
    g = run_gpu(s, precision="fp16")
    a = run_gpu(s, precision="fp32")
    e, e32 = errors(g, ref), errors(a, ref)
    print(f"fp16 p={p}: {e}; fp32: {e32}")
    assert g["status"] == 0
    for k in ("E", "F", "dVdl"):
        assert e[k] < 1.05 * e32[k] + 1e-6, (k, e, e32)


def test_fp16_close_to_fp32_path():
    """The FP16 form against the FP32 CUDA-core path on the same input: the degrees 0..3 of
    every multipole carry about 2^-22 relative rounding, the higher degrees 2^-12 of terms
    that are themselves small.  Measured bars as for the split BF16 form; a wrong cell
    layout, chunk kind or descriptor shows as an O(1) difference."""
    s = synth.periodic_uniform(seed=11, n=6000, L=3.5, n_sites=8, site_size=4, p=10, depth=3)
    a = run_gpu(s, precision="fp32")
    b = run_gpu(s, precision="fp16")
    dF = np.sqrt(((a["F"] - b["F"]) ** 2).sum() / (a["F"] ** 2).sum())
    dE = abs(a["E"] - b["E"]) / abs(a["E"])
    dV = np.linalg.norm(a["dVdl"] - b["dVdl"]) / np.linalg.norm(a["dVdl"])
    print(f"fp16 vs fp32: dF {dF:.2e} dE {dE:.2e} dVdl {dV:.2e}")
    assert dF < 2e-6 and dE < 1e-5 and dV < 1e-4, (dF, dE, dV)


@pytest.mark.parametrize("precision", ["fp16", "3xbf16"])
def test_kernel_tiles_give_identical_results(precision):
    """The M2L tile width (128, 160, 192, 224, 256 rows per CTA) and the near-field block shape (1, 2 or
    4 leaves per block) only change how the work is split: every choice gives bit for bit the
    result of the default, at depths 3 and 5."""
    from paper_2410_01626_b300 import FMM
    for s in (synth.periodic_uniform(seed=17, n=40000, L=5.0, n_sites=8, site_size=4, p=10, depth=3),
              synth.periodic_uniform(seed=18, n=150000, L=10.0, n_sites=8, site_size=4, p=10, depth=5)):
        d = to_dev(s)
        outs = []
        for rows, warps in ((0, 0), (128, 0), (160, 0), (224, 0), (256, 0), (0, 2), (128, 4), (0, 1)):
            f = FMM(s["L"], True, s["p"], s["depth"], precision=precision, m2l_rows=rows, p2p_warps=warps)
            f.set_charges(d["qA"], d["qB"], d["site"], d["lam"])
            E, F, dV, phi = f.eval(d["x"], phi=True)
            torch.cuda.synchronize()
            assert f.status_word() == 0
            outs.append((E.item(), F.cpu(), dV.cpu(), phi.cpu()))
            f.close()
        for o in outs[1:]:
            assert o[0] == outs[0][0]
            for a, b in zip(o[1:], outs[0][1:]):
                assert torch.equal(a, b)
    from paper_2410_01626_b300 import FmmError
    with pytest.raises(FmmError):
        FMM(3.0, True, 8, 3, precision=precision, m2l_rows=100)
    with pytest.raises(FmmError):
        FMM(3.0, True, 8, 3, precision=precision, p2p_warps=8)
