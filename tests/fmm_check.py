"""Shared helpers of the GPU parity tests: run the CUDA path on a synthetic
system and compare it with the FP64 oracle.

Error metrics (relative): E |dE|/|E|; F sqrt(sum |dF|^2 / sum |F|^2) over the
compared atoms; dV/dlambda ||d||_2 / ||ref||_2 over sites.
"""
import hashlib

import numpy as np
import torch

import oracle
from paper_2410_01626_b300 import FMM


def to_dev(s, dev="cuda"):
    return {
        "x": torch.from_numpy(np.ascontiguousarray(s["x"])).to(dev),
        "qA": torch.from_numpy(s["qA"]).to(dev),
        "qB": torch.from_numpy(s["qB"]).to(dev),
        "site": torch.from_numpy(s["site"]).to(dev),
        "lam": torch.from_numpy(s["lam"]).to(dev),
    }


def make_solver(s, p=None, depth=None, precision="fp32", interpolation="charge"):
    f = FMM(s["L"], s["periodic"], s["p"] if p is None else p, s["depth"] if depth is None else depth,
            origin=s["origin"], precision=precision, interpolation=interpolation)
    d = to_dev(s)
    f.set_charges(d["qA"], d["qB"], d["site"], d["lam"])
    return f, d


def run_gpu(s, p=None, depth=None, precision="fp32", interpolation="charge"):
    f, d = make_solver(s, p, depth, precision, interpolation)
    E, F, dV, phi = f.eval(d["x"], phi=True)
    torch.cuda.synchronize()
    st = f.status_word()
    out = {"E": float(E.item()), "F": F.cpu().numpy().astype(np.float64), "dVdl": dV.cpu().numpy().astype(np.float64),
           "phi": phi.cpu().numpy().astype(np.float64), "status": st}
    f.close()
    return out


def errors(gpu, ref, idx=None):
    e = {}
    if "E" in ref:
        e["E"] = abs(gpu["E"] - ref["E"]) / abs(ref["E"])
    Fg = gpu["F"] if idx is None else gpu["F"][idx]
    Fr = ref["F"]
    e["F"] = float(np.sqrt(((Fg - Fr) ** 2).sum() / (Fr ** 2).sum()))
    if len(ref["dVdl"]):
        e["dVdl"] = float(np.linalg.norm(gpu["dVdl"] - ref["dVdl"]) / np.linalg.norm(ref["dVdl"]))
    return e


_cache = {}


def system_digest(s):
    h = hashlib.sha1()
    for k in ("x", "qA", "qB", "site", "lam"):
        h.update(np.ascontiguousarray(s[k]).tobytes())
    h.update(repr((s["L"], s["origin"], s["periodic"])).encode())
    return h.hexdigest()


def oracle_ref(s, targets=None, tol=1e-11, hamiltonian=False):
    t = None if targets is None else hashlib.sha1(np.asarray(targets, np.int64).tobytes()).hexdigest()
    k = (system_digest(s), t, tol, hamiltonian)
    if k not in _cache:
        _cache[k] = oracle.evaluate(s, targets=targets, tol=tol, hamiltonian=hamiltonian)
    return _cache[k]
