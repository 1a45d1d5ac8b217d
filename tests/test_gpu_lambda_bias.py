"""Biased lambda dynamics on the GPU (double well, pH potential, partition function
correction; Sec. 2.2-2.3): the force against the oracle's potential, and the sampled
protonation fractions against the Henderson-Hasselbalch ratio the correction targets."""
import math

import numpy as np
import pytest
import torch

from oracle import lambda_bias as lb
from paper_2410_01626_b300 import lambda_bias, lambda_step

pytestmark = pytest.mark.gpu
KT = 2.494339


def test_double_well_force_matches_oracle():
    """gamma = 0, kT = 0, v = 0, first step: lambda_1 - lambda_0 = dt^2 f / (2 m) exactly
    (no noise, no friction), so f is recovered and compared with -dV_dw/dlambda.  A long
    step (0.02 ps) makes the displacement large against the FP32 rounding of lambda (two
    half drifts, at most one ulp = 1.2e-7 near lambda = 1); starts stay clear of the walls."""
    n = 2048
    rng = np.random.default_rng(0)
    l0 = rng.uniform(-0.08, 1.08, n).astype(np.float32)
    pk = rng.uniform(2.0, 6.0, n)
    bias = lambda_bias(4.0, pk, 6.0, KT)
    lam = torch.from_numpy(l0).cuda()
    vel = torch.zeros(n, device="cuda")
    zero = torch.zeros(n, device="cuda")
    dt, m = 0.02, 60.0
    lambda_step(lam, vel, zero, step=0, seed=1, dt=dt, mass=m, gamma=0.0, kT=0.0, first=True, bias=bias)
    f = 2 * m * (lam.double().cpu().numpy() - l0.astype(np.float64)) / dt ** 2
    b = bias.double().cpu().numpy()
    want = np.array([-lb.potential(float(x), *row)[1] for x, row in zip(l0, b)])
    scale = np.abs(want).max()
    assert np.abs(f - want).max() < 1e-4 * scale + 2 * m * 1.2e-7 / dt ** 2


def test_sampled_protonation_matches_the_corrected_populations():
    """8192 independent lambda particles in the corrected double well at four pH - pKa
    values.  The correction (Sec. 2.3) sets the offset from the partition functions over
    [0, 0.5] and [0.5, 1]; the dynamics samples the whole interval between its reflecting
    walls (-0.1, 1.1), harmonic walls included.  So the fraction with lambda > 0.5
    approaches r / (1 + r), r = Z_deprot / Z_prot of the corrected potential over the walls'
    interval (oracle quadrature); r is 10^(pH - pKa) only up to the walls' tails.
    A light particle (5 u), gamma = 2 / ps and a 2 kJ/mol barrier keep the well-to-well
    transition time (Kramers) near 3 ps, so 60 ps gives ~20 transitions per particle."""
    groups = [-1.0, 0.0, 0.5, 1.5]
    per = 2048
    n = per * len(groups)
    pH, barrier = 5.0, 2.0
    pk = np.repeat([pH - g for g in groups], per)
    bias = lambda_bias(pH, pk, barrier, KT)
    lam = torch.full((n,), 0.5, device="cuda")
    vel = torch.zeros(n, device="cuda")
    zero = torch.zeros(n, device="cuda")
    frac = torch.zeros(len(groups), dtype=torch.float64, device="cuda")
    samples = 0
    for step in range(30000):
        lambda_step(lam, vel, zero, step=step, seed=7, dt=0.002, mass=5.0, gamma=2.0, kT=KT, first=step == 0,
                    bias=bias)
        if step >= 2500 and step % 10 == 0:
            frac += (lam > 0.5).view(len(groups), per).double().mean(1)
            samples += 1
    frac = (frac / samples).cpu().numpy()
    for g, fr in zip(groups, frac):
        d = lb.pfc_delta(pH=pH, pKa=pH - g, h=barrier, kT=KT)
        r = lb.population_ratio(0.0, 1.0, barrier, d, 1000.0, KT, lo=-0.1, hi=1.1)
        assert fr == pytest.approx(r / (1 + r), abs=0.015), (g, fr, r / (1 + r))
