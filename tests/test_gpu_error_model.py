"""The GPU results follow the paper's error model (Sec. 4, Eq. 4.3 and 4.6).

Protocol of Sec. 4 on the GPU: uniform random charges for (L, N, xi L)
drawn from the paper's grid of cases, a grid fine enough that the Fourier
truncation is negligible, and P from 4 upward.  The rms potential error
against the direct Ewald k-space sum (O1), scaled by A_P = sqrt(Q xi L)/L,
lies in [0.1, 1] x e^{-pi P c^2/2}; the rms force error scaled by
A_F = 4 pi Q sqrt(xi^3 / L) lies below e^{-pi P c^2/2}.  Checked for the FP64
path and, where the bound is far above single-precision rounding, for the
single-precision pipeline.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1712_04718_gb300 import se, systems

pytestmark = pytest.mark.gpu

C_SHAPE = 0.95


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


CASES = [(1.0, 200, 5.0), (5.0, 400, 15.0), (10.0, 800, 15.0), (20.0, 1200, 25.0)]


@pytest.mark.parametrize("L,N,xiL", CASES)
def test_scaled_errors_follow_eq_4_6(L, N, xiL):
    xi = xiL / L
    x, q = systems.uniform_charges(N, L, seed=7 * N + int(L))
    Q = float((q ** 2).sum())
    _, phio, Fo = oracle.ewald_kspace(x, q, L, xi)
    M = 2 * math.ceil(6.1 * xi * L / math.pi)
    AP = math.sqrt(Q * xi * L) / L
    AF = 4 * math.pi * Q * math.sqrt(xi ** 3 / L)
    for prec, Ps in (("fp64", (4, 8, 12, 16)), ("fp32", (4, 6, 8))):
        dt = torch.float64 if prec == "fp64" else torch.float32
        xd = torch.tensor(x, dtype=dt, device="cuda")
        qd = torch.tensor(q, dtype=dt, device="cuda")
        for P in Ps:
            if P > M:
                continue
            plan = se.Plan(N, L, xi, M, P, precision=prec)
            _, F, phi = plan.energy_force(xd, qd)
            plan.close()
            b = math.exp(-math.pi * P * C_SHAPE ** 2 / 2)
            ep = math.sqrt(((phi.double().cpu().numpy() - phio) ** 2).mean()) / AP
            ef = math.sqrt(((F.double().cpu().numpy() - Fo) ** 2).sum(1).mean()) / AF
            assert 0.1 * b < ep < b, (prec, P, ep / b)
            assert ef < b, (prec, P, ef / b)
