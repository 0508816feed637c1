"""se_spread_noalloc: the spreading step for callers that cannot allocate
device memory (for example a program that reserves all of its GPU memory at
start-up and forbids allocation in its time-step loop, or a component whose
device memory belongs to another framework's allocator).

The entry point keeps its scratch in a fixed device array and writes into a
grid the caller owns.  This test calls it through the C ABI and checks its
grid against the plan-based se_spread (which allocates its own buffers), on
several calls in a row, with the FP64 tolerance of the other parity tests.
It lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1712_04718_gb300 import _native as nat
from paper_1712_04718_gb300 import se, systems

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


# (N, M, P): the 32 768-particle limit on the largest grid (4096 tiles, the
# scratch's tile bound), a grid that is not a multiple of the tile edge
# (partial edge tiles), and a support whose region exceeds the shared-memory
# budget of one pass (the tiled spread works in slabs)
SHAPES = [(2000, 32, 8), (32768, 128, 8), (3000, 50, 6), (2000, 48, 24)]


@pytest.mark.parametrize("N,M,P", SHAPES)
def test_spread_noalloc_matches_plan_spread(N, M, P):
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    lib = nat.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = 3.0
    # xi so that eta = P L^2 xi^2 / (c^2 pi M^2) stays at 0.5 (Eq. 4.2)
    xi = min(3.5, (0.5 * 0.95 ** 2 * np.pi * M * M / (P * L * L)) ** 0.5)
    # three calls in a row: the scratch keeps the previous call's contents,
    # so a repeated input and a new input must both come out right
    for seed in (3, 3, 4):
        x, q = systems.uniform_charges(N, L, seed=seed + M)
        xd = torch.tensor(x, device="cuda")
        qd = torch.tensor(q, device="cuda")
        H = torch.full((M, M, M), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.se_spread_noalloc(_p(xd), _p(qd), N, L, xi, M, P, _p(H), stream)
        assert rc == nat.SE_OK, nat.strerror(rc)
        plan = se.Plan(N, L, xi, M, P, precision="fp64")
        plan.spread(xd, qd)
        Href = plan.copy_grid(0)
        torch.cuda.synchronize()
        assert torch.isfinite(H).all()
        assert _rel(H, Href) < TOL_FP64
        plan.close()
