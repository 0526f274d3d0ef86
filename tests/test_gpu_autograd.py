"""The band-energy gradient through torch.autograd (ALBBandEnergy) on the GPU path (FP64).

Checks that the backward pass returns what dgdft_alb_grad forms, that it matches the oracle's
Hellmann-Feynman gradient, and that it matches central finite differences of the GPU energy itself
in one atom coordinate (step 1e-4 bohr: truncation error O(1e-8) relative) and along one seeded
direction of V_eff (step 1e-5 Ha).
"""
import numpy as np
import pytest
import torch

from oracle import driver
from workloads.configs import make_slab, probe_directions
from gpu_util import gpu_context

pytestmark = pytest.mark.gpu

OPTS = dict(precision=0, cheb_degree=12, tol=1e-11, max_iter=400)


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


def _case():
    w = make_slab(2, 1, (6, 10, 10), (10, 10, 10), 0.5, 8, 4, 17, width=0.6, proj_width=0.6,
                  r_cut=2.4, lattice=1, jitter=0.5, zjitter=0.4)
    w.problem.v_extra = np.random.default_rng(8).normal(size=w.problem.v_extra.size) * 0.05
    w.n_electrons = np.array([4.0, 4.0])
    w.kT = 0.02
    return w


def _energy(ctx, w, v, R):
    from paper_2003_00407_gb300.api import ALBBandEnergy
    return ALBBandEnergy.apply(v, R, ctx, w.problem, w.params, w.kT, w.n_electrons, OPTS)


def test_backward_is_the_adjoint_gradient(ctx):
    from paper_2003_00407_gb300 import api
    w = _case()
    p, q = w.problem, w.params
    v = torch.tensor(p.v_extra, dtype=torch.float64, device="cuda", requires_grad=True)
    R = torch.tensor(p.atom_pos, dtype=torch.float64, requires_grad=True)
    E = _energy(ctx, w, v, R)
    E.backward()
    res = api.alb_generate(ctx, p, q, **OPTS)
    E2, gv, gR = api.alb_grad(ctx, p, q, res, w.kT, w.n_electrons)
    assert abs(E.detach().item() - float(E2.sum())) <= 1e-10
    assert torch.allclose(v.grad, gv, rtol=0, atol=1e-12)
    assert torch.allclose(R.grad, gR.cpu(), rtol=0, atol=1e-12)
    sols = {k: driver.solve_element(p, q, k, dense_route=True) for k in range(p.n_elem)}
    E_o, gv_o, gR_o = driver.alb_grad(p, sols, w.kT, w.n_electrons)
    assert abs(E.detach().item() - E_o.sum()) <= 1e-8
    assert np.abs(R.grad.numpy() - gR_o).max() <= 1e-7 * max(1.0, np.abs(gR_o).max())
    assert np.abs(v.grad.cpu().numpy() - gv_o).max() <= 1e-7 * max(1.0, np.abs(gv_o).max())


def test_backward_matches_central_differences(ctx):
    w = _case()
    p = w.problem
    v0 = torch.tensor(p.v_extra, dtype=torch.float64, device="cuda")
    R0 = torch.tensor(p.atom_pos, dtype=torch.float64)
    v = v0.clone().requires_grad_(True)
    R = R0.clone().requires_grad_(True)
    _energy(ctx, w, v, R).backward()
    h = 1e-4
    worst = 0.0
    for (ia, ax) in [(0, 0), (1, 2)]:
        Rp, Rm = R0.clone(), R0.clone()
        Rp[ia, ax] += h
        Rm[ia, ax] -= h
        with torch.no_grad():
            fd = (float(_energy(ctx, w, v0, Rp)) - float(_energy(ctx, w, v0, Rm))) / (2 * h)
        g = float(R.grad[ia, ax])
        worst = max(worst, abs(fd - g))
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (ia, ax, fd, g)
    d = torch.tensor(probe_directions(1, v0.numel(), 99)[0], dtype=torch.float64, device="cuda")
    hv = 1e-5
    with torch.no_grad():
        fd = (float(_energy(ctx, w, v0 + hv * d, R0)) - float(_energy(ctx, w, v0 - hv * d, R0))) / (2 * hv)
    g = float(torch.dot(v.grad, d))
    assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (fd, g)
    print("finite differences: worst atom-coordinate difference", worst, "V direction", abs(fd - g))
