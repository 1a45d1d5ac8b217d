"""Device-side lambda dynamics and batched replicas."""
import math

import numpy as np
import pytest
import torch

import synth
from fmm_check import make_solver, to_dev
from paper_2410_01626_b300 import FMM, Batch, lambda_step
from philox_ref import philox4x32_10

pytestmark = pytest.mark.gpu


def test_lambda_step_noise_is_philox_box_muller():
    """With zero force and zero velocity, one step leaves v = c2 * xi with xi the Box-Muller
    normal of Philox4x32-10(counter = (step, 0, site, 0), key = seed)."""
    K = 64
    lam = torch.full((K,), 0.5, device="cuda")
    vel = torch.zeros(K, device="cuda")
    dV = torch.zeros(K, device="cuda")
    seed, step, dt, m, g, kT = 0x1234567890ABCDEF, 77, 0.002, 60.0, 1.0, 2.494339
    lambda_step(lam, vel, dV, step, seed, dt=dt, mass=m, gamma=g, kT=kT, first=True, lo=-10.0, hi=10.0)
    v = vel.cpu().numpy().astype(np.float64)
    c1 = math.exp(-g * dt)
    c2 = math.sqrt((1 - c1 * c1) * kT / m)
    for k in range(K):
        r = philox4x32_10((step & 0xFFFFFFFF, step >> 32, k, 0), (seed & 0xFFFFFFFF, seed >> 32))
        u1 = ((r[0] >> 8) + 1) / 16777216.0
        u2 = ((r[1] >> 8) + 1) / 16777216.0
        xi = math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
        assert v[k] == pytest.approx(c2 * xi, rel=1e-5, abs=1e-6)


def _loop(f, d, lam0, steps, seed, start=0, vel0=None):
    """`steps` lambda steps start .. start+steps-1: eval (CUDA graph after the first, eager,
    step), then one device Langevin step; returns lambda after every step."""
    lam = lam0.clone()
    vel = torch.zeros_like(lam) if vel0 is None else vel0.clone()
    f.bind_lambda(lam)
    E, F, dV, _ = f.outputs()
    traj = []
    g = None
    for s in range(start, start + steps):
        if g is None:
            f.eval_into(d["x"], E, F, dV)
            g = torch.cuda.CUDAGraph()
            stream = torch.cuda.Stream()
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                with torch.cuda.graph(g, stream=stream):
                    f.eval_into(d["x"], E, F, dV)
            torch.cuda.current_stream().wait_stream(stream)
        else:
            g.replay()
        lambda_step(lam, vel, dV, s, seed, first=(s == 0))
        traj.append(lam.clone())
    torch.cuda.synchronize()
    f.bind_lambda(None)
    return torch.stack(traj), lam, vel


def test_lambda_dynamics_loop_bounded_deterministic_resumable():
    s = synth.periodic_uniform(seed=12, n=6000, L=4.0, n_sites=16, site_size=4, p=8, depth=3)
    f, d = make_solver(s, precision="3xtf32")
    lam0 = d["lam"].clone()
    t1, lam1, vel1 = _loop(f, d, lam0, 120, seed=5)
    t2, _, _ = _loop(f, d, lam0, 120, seed=5)
    assert torch.equal(t1, t2)                       # deterministic
    assert (t1 >= -0.1).all() and (t1 <= 1.1).all()  # reflecting walls
    assert (t1[-1] != t1[0]).any()                   # it moves
    # resume: 60 steps, checkpoint (lambda, velocity, step), 60 more == 120 in one go
    ta, lam_a, vel_a = _loop(f, d, lam0, 60, seed=5)
    tb, _, _ = _loop(f, d, lam_a, 60, seed=5, start=60, vel0=vel_a)
    assert torch.equal(torch.cat([ta, tb]), t1)
    f.close()


def test_batch_equals_standalone_bitwise():
    systems = [synth.replica(100 + i) for i in (0, 3, 7, 12)]
    systems += [synth.periodic_uniform(seed=21, n=3000, L=3.0, p=8, depth=3),
                synth.open_uniform(seed=22, n=2500, L=4.0, n_sites=3, site_size=4, p=6, depth=3)]
    precisions = ["3xtf32", "tf32", "fp32", "3xbf16", "fp16", "3xbf16"]
    solvers, devs, refs = [], [], []
    for s, prec in zip(systems, precisions):
        f, d = make_solver(s, precision=prec)
        E, F, dV, _ = f.eval(d["x"])
        solvers.append(f)
        devs.append(d)
        refs.append((E.clone(), F.clone(), dV.clone()))
    torch.cuda.synchronize()
    outs = [f.outputs() for f in solvers]
    b = Batch(solvers)
    for _ in range(2):  # capture, then a replay of the same graph
        for o in outs:
            o[0].zero_(); o[1].zero_(); o[2].zero_()
        b.eval_into([d["x"] for d in devs], [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o[0], r[0]) and torch.equal(o[1], r[1]) and torch.equal(o[2], r[2])
    b.close()
    for f in solvers:
        f.close()


def test_handles_of_different_depths_coexist():
    """A deeper handle created first must still evaluate after a shallower one was created
    (per-kernel launch limits are process wide)."""
    deep = synth.periodic_uniform(seed=30, n=20000, L=5.0, p=8, depth=4)
    shallow = synth.periodic_uniform(seed=31, n=3000, L=3.0, p=8, depth=3)
    f1, d1 = make_solver(deep, precision="3xtf32")
    E1, F1, dV1, _ = f1.eval(d1["x"])
    f2, d2 = make_solver(shallow, precision="3xtf32")
    f2.eval(d2["x"])
    E1b, F1b, dV1b, _ = f1.eval(d1["x"])
    torch.cuda.synchronize()
    assert torch.equal(E1, E1b) and torch.equal(F1, F1b)
    f1.close()
    f2.close()
