"""GPU parity of the band-energy gradient (dgdft_alb_grad) against the oracle (FP64 path)."""
import numpy as np
import pytest
import torch

from oracle import driver
from workloads.configs import make_slab
from gpu_util import gpu_context

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("precision", [0, 1])
def test_gradient_matches_oracle(ctx, precision):
    from paper_2003_00407_gb300 import api
    w = _case()
    p, q = w.problem, w.params
    sols = {k: driver.solve_element(p, q, k, dense_route=True) for k in range(p.n_elem)}
    E_o, gv_o, gR_o = driver.alb_grad(p, sols, w.kT, w.n_electrons)
    res = api.alb_generate(ctx, p, q, precision=precision, cheb_degree=12, tol=1e-11, max_iter=400)
    E, gv, gR = api.alb_grad(ctx, p, q, res, w.kT, w.n_electrons)
    E, gv, gR = E.cpu().numpy(), gv.cpu().numpy(), gR.cpu().numpy()
    tol = 1e-8 if precision == 0 else 1e-5
    assert np.abs(E - E_o).max() <= tol * 10
    assert np.abs(gv - gv_o).max() <= tol * max(1.0, np.abs(gv_o).max())
    assert np.abs(gR - gR_o).max() <= tol * max(1.0, np.abs(gR_o).max()), (gR, gR_o)
