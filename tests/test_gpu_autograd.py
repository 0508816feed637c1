"""The differentiable SE energy (autograd Function over se_adjoint).

Checks: backward equals the analytic force and potential of the same plan;
central finite differences (h = 1e-4 nm) of the FP64 GPU energy on 32 atoms
of the 100 200-atom water box, screened so that x +- h stays in the same grid
cell (the truncated window jumps at cell faces); the FP32 gradient against
the FP64 one and against the oracle's analytic gradient; the recompute path.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1712_04718_gb300 import se, systems
from paper_1712_04718_gb300.autograd import se_energy
from parity import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)




@pytest.mark.parametrize("prec,tol,variant", [("fp64", 1e-13, 0), ("fp32", 1e-6, 0),
                                              ("fp32", 1e-6, 5)])
def test_backward_is_force_and_potential(prec, tol, variant):
    L, xi, M, P = 2.0, 4.0, 24, 8
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x, q = systems.uniform_charges(300, L, seed=31)
    plan = se.Plan(len(q), L, xi, M, P, precision=prec, spread_variant=variant)
    xd = torch.tensor(x, dtype=dtype, device="cuda")
    qd = torch.tensor(q, dtype=dtype, device="cuda")
    E0, F, phi = plan.energy_force(xd, qd)
    xg = xd.clone().requires_grad_(True)
    qg = qd.clone().requires_grad_(True)
    E = se_energy(xg, qg, plan)
    assert abs(E.item() - E0) < (1e-12 if prec == "fp64" else 1e-6) * abs(E0)
    g = 2.5
    (g * E).backward()
    assert_close(xg.grad.double().cpu(), (-g * F).double().cpu(), tol)
    assert_close(qg.grad.double().cpu(), (g * phi).double().cpu(), tol)
    plan.close()


def _same_cell_atoms(x, h_grid, step, count, rng):
    frac = x / h_grid - np.floor(x / h_grid)
    ok = np.all((frac > step / h_grid * 1.01) & (frac < 1 - step / h_grid * 1.01), axis=1)
    idx = np.flatnonzero(ok)
    return rng.choice(idx, size=count, replace=False)


def test_finite_differences_fp64_water_100k():
    """Central differences of the FP64 GPU energy equal the backward gradient."""
    x, q, w = systems.make("water-L10-M84-P8-fp32comp", dtype=np.float64)
    plan = se.Plan(len(q), w["L"], w["xi"], w["M"], w["P"], precision="fp64")
    xd = torch.tensor(x, device="cuda")
    qd = torch.tensor(q, device="cuda")
    xg = xd.clone().requires_grad_(True)
    E = se_energy(xg, qd, plan)
    E.backward()
    grad = xg.grad.cpu().numpy()
    h = 1e-4
    rng = np.random.default_rng(4)
    atoms = _same_cell_atoms(x, w["L"] / w["M"], h, 32, rng)
    fd = np.zeros((len(atoms), 3))
    Ebuf = torch.zeros(1, dtype=torch.float64, device="cuda")
    for i, m in enumerate(atoms):
        for d in range(3):
            vals = []
            for s in (+1, -1):
                xs = xd.clone()
                xs[m, d] += s * h
                plan.spread(xs, qd)
                plan.scale(Ebuf)
                vals.append(Ebuf.item())
            fd[i, d] = (vals[0] - vals[1]) / (2 * h)
    err = np.abs(fd - grad[atoms]).max()
    scale = np.abs(grad[atoms]).max()
    assert err < 1e-5 * max(scale, 1.0), (err, scale)
    plan.close()


def test_fp32_gradient_against_fp64_and_oracle():
    """The FP32 (single-precision pipeline) gradient of the 100k-atom box
    against the FP64 GPU gradient, and against the oracle's analytic force
    (dE/dx = -F of the plain CPU SE, the cell decisions in float32)."""
    x, q, w = systems.make("water-L10-M84-P8-fp32comp")
    N = len(q)
    grads = {}
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec)
        xg = torch.tensor(x, dtype=dt, device="cuda").requires_grad_(True)
        qg = torch.tensor(q, dtype=dt, device="cuda").requires_grad_(True)
        se_energy(xg, qg, plan).backward()
        grads[prec] = (xg.grad.double().cpu().numpy(), qg.grad.double().cpu().numpy())
        plan.close()
    # per-particle outputs of the single-precision pipeline: 5 x 2e-5, the
    # bound of every FP32 particle comparison (2e-5 is the grids' bound)
    assert_close(grads["fp32"][0], grads["fp64"][0], 1e-4, q=q, label="dE/dx")
    assert_close(grads["fp32"][1], grads["fp64"][1], 1e-4, label="dE/dq")
    r = oracle.se_kspace(np.asarray(x, np.float64), np.asarray(q, np.float64), w["L"], w["xi"],
                         w["M"], w["P"], cell_mode=32)
    assert_close(grads["fp32"][0], -r["F"], 1e-4, q=q, label="dE/dx vs oracle")
    assert_close(grads["fp32"][1], r["phi"], 1e-4, label="dE/dq vs oracle")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_recompute_when_grid_overwritten(prec):
    """Two forwards on one plan, then backward of the first: the grid of the
    first is gone and is recomputed; recompute=True always recomputes."""
    L, xi, M, P = 2.0, 4.0, 20, 6
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x, q = systems.uniform_charges(200, L, seed=33)
    x2, q2 = systems.uniform_charges(200, L, seed=34)
    plan = se.Plan(200, L, xi, M, P, precision=prec)
    ref = se.Plan(200, L, xi, M, P, precision=prec)
    xa = torch.tensor(x, dtype=dtype, device="cuda").requires_grad_(True)
    qa = torch.tensor(q, dtype=dtype, device="cuda")
    xb = torch.tensor(x2, dtype=dtype, device="cuda").requires_grad_(True)
    qb = torch.tensor(q2, dtype=dtype, device="cuda")
    Ea = se_energy(xa, qa, plan)
    Eb = se_energy(xb, qb, plan)
    Ea.backward()
    _, F, _ = ref.energy_force(xa.detach(), qa)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert_close(xa.grad.double().cpu(), -F.double().cpu(), tol)
    xc = torch.tensor(x, dtype=dtype, device="cuda").requires_grad_(True)
    se_energy(xc, qa, plan, recompute=True).backward()
    assert_close(xc.grad.double().cpu(), -F.double().cpu(), tol)
    plan.close()
    ref.close()


def test_graph_captured_forward_and_backward():
    """The differentiable energy's forward and backward captured in one CUDA
    graph (static inputs) and replayed: the gradients equal the eager ones,
    and a replay after the positions change in place follows them."""
    x, q, w = systems.make("water-L6-M52-P8-fp32comp")
    N = len(q)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision="fp32")
    xg = torch.tensor(x, device="cuda").requires_grad_(True)
    qg = torch.tensor(q, device="cuda").requires_grad_(True)
    se_energy(xg, qg, plan).backward()
    gx0, gq0 = xg.grad.clone(), qg.grad.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            xg.grad = None
            qg.grad = None
            se_energy(xg, qg, plan).backward()
    torch.cuda.current_stream().wait_stream(s)
    xg.grad = None
    qg.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        E = se_energy(xg, qg, plan)
        E.backward()
    g.replay()
    torch.cuda.synchronize()
    assert_close(xg.grad.double().cpu(), gx0.double().cpu(), 1e-6, q=q)
    assert_close(qg.grad.double().cpu(), gq0.double().cpu(), 1e-6)
    with torch.no_grad():
        xg += 0.01
    g.replay()
    torch.cuda.synchronize()
    F = torch.empty((N, 3), device="cuda")
    plan.evaluate(xg.detach(), qg.detach(), F)
    torch.cuda.synchronize()
    assert_close(xg.grad.double().cpu(), -F.double().cpu(), 1e-6, q=q)
    plan.close()
