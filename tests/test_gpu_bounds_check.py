"""The bounds-checked build (libfmmcph_checked.so, compiled with -DFMM_BOUNDS_CHECK).

The data-dependent indices of the kernels are checked against their extents in that build. These
are the leaf keys, sorted slots, permutation entries, leaf ranges, site atoms, staged-buffer
offsets, and packed-box and operator indices. A failed check skips the access it guards, and
fmm_status_word reports it as FMM_DEV_BOUNDS, with the file and line in fmm_last_error.

A child process loads that build (FMMCPH_BOUNDS_CHECK=1). It evaluates small systems of at most
64 atoms at depth <= 2, open and periodic, in every precision form and both interpolations. It
also evaluates one system whose leaves exceed the near field's 64-target tile. Each evaluation
must:
- report no failed check;
- repeat bitwise (eager, captured, replayed);
- equal bitwise what the normal build computes in this process, since the checks change no
  arithmetic;
- match the FP64 oracle.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synth
from fmm_check import errors, make_solver, oracle_ref
from paper_2410_01626_b300 import binding

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    ("open64_fp32", "open_uniform", dict(seed=60, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=2), "fp32", "charge"),
    ("open64_fp16", "open_uniform", dict(seed=60, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=2), "fp16", "charge"),
    ("per64_fp16", "periodic_uniform", dict(seed=61, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=2), "fp16",
     "charge"),
    ("per64_3xbf16", "periodic_uniform", dict(seed=61, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=2), "3xbf16",
     "charge"),
    ("per64_tf32", "periodic_uniform", dict(seed=61, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=2), "tf32",
     "charge"),
    ("per64_fp32_ham", "periodic_uniform", dict(seed=62, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=2), "fp32",
     "hamiltonian"),
    ("per64_d1_fp16", "periodic_uniform", dict(seed=63, n=64, L=2.0, n_sites=4, site_size=4, p=8, depth=1), "fp16",
     "charge"),
    ("open500_d1_items", "open_uniform", dict(seed=64, n=500, L=3.0, n_sites=4, site_size=4, p=4, depth=1), "fp32",
     "charge"),
]

# the child: loads the checked build, evaluates every case three times, saves the first result
CHILD = r"""
import json, os, sys
import numpy as np
root, out = sys.argv[1], sys.argv[2]
sys.path[:0] = [root, os.path.join(root, "tests")]
import torch
import synth
from paper_2410_01626_b300 import binding
from fmm_check import make_solver
lib = binding.load()
res = {"flags": int(lib.fmm_build_flags()), "path": binding.library_path(), "cases": {}}
for name, gen, kw, precision, interp in json.loads(sys.argv[3]):
    s = getattr(synth, gen)(**kw)
    f, d = make_solver(s, precision=precision, interpolation=interp)
    runs, status = [], []
    for _ in range(3):  # eager, then captured, then replayed
        E, F, dV, phi = f.eval(d["x"], phi=True)
        torch.cuda.synchronize()
        status.append(f.status_word())
        runs.append((float(E.item()), F.cpu().numpy(), dV.cpu().numpy(), phi.cpu().numpy()))
    f.close()
    same = all(r[0] == runs[0][0] and all(np.array_equal(a, b) for a, b in zip(r[1:], runs[0][1:])) for r in runs)
    np.savez(os.path.join(out, name + ".npz"), E=runs[0][0], F=runs[0][1], dV=runs[0][2], phi=runs[0][3])
    res["cases"][name] = {"status": status, "repeat_bitwise": bool(same),
                          "last_error": lib.fmm_last_error().decode()}
print(json.dumps(res))
"""


@pytest.fixture(scope="module")
def checked_run(tmp_path_factory):
    out = tmp_path_factory.mktemp("bounds")
    env = dict(os.environ, FMMCPH_BOUNDS_CHECK="1")
    spec = json.dumps([list(c) for c in CASES])
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out), spec], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), out


def test_child_loaded_the_checked_build(checked_run):
    res, _ = checked_run
    assert res["flags"] & 1, res
    assert res["path"].endswith("libfmmcph_checked.so"), res["path"]
    assert binding.load().fmm_build_flags() == 0  # this process: the normal build


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_checked_build_no_failed_check_and_equal_to_normal_build(checked_run, case):
    res, out = checked_run
    name, gen, kw, precision, interp = case
    r = res["cases"][name]
    assert r["status"] == [0, 0, 0], r  # no FMM_DEV_BOUNDS (8), nor any other bit
    assert r["repeat_bitwise"], r
    c = np.load(os.path.join(str(out), name + ".npz"))
    s = getattr(synth, gen)(**kw)
    f, d = make_solver(s, precision=precision, interpolation=interp)
    E, F, dV, phi = f.eval(d["x"], phi=True)
    torch.cuda.synchronize()
    assert f.status_word() == 0
    f.close()
    assert float(E.item()) == float(c["E"])
    np.testing.assert_array_equal(F.cpu().numpy(), c["F"])
    np.testing.assert_array_equal(dV.cpu().numpy(), c["dV"])
    np.testing.assert_array_equal(phi.cpu().numpy(), c["phi"])
    ref = oracle_ref(s, hamiltonian=interp == "hamiltonian", tol=1e-10)
    g = {"E": float(c["E"]), "F": c["F"].astype(np.float64), "dVdl": c["dV"].astype(np.float64)}
    e = errors(g, ref)
    tol = 5e-3 if precision == "tf32" or kw["p"] < 8 else 1e-3  # TF32 operands; truncation at order p
    assert e["E"] < tol and e["F"] < tol and e["dVdl"] < tol, e
