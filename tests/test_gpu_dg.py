"""GPU parity of the DG assembly (Eq. DGHamiltonian) against the oracle.

ALB bases from the GPU and the oracle may differ by an orthogonal rotation
W_k = A_o,k A_g,k^T dV inside each element, so blocks are compared as
W_k H^g_{kn} W_n^T against H^o_{kn} (contract 1e-6 Ha), and the lowest
eigenvalues of the assembled dense H^DG directly.
"""
import numpy as np
import pytest
import torch

from oracle import driver, dg as odg
from workloads.configs import make_slab
from workloads.problem import STENCIL_XY9
from gpu_util import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


def _compare(w, blocks_g, A_g, sols, alpha, tol=1e-6):
    p, q = w.problem, w.params
    ingr = [odg.element_ingredients(p, k, sols[k]["X"][:sols[k]["n_eig"]], sols[k]["C"], sols[k]["A"])
            for k in range(p.n_elem)]
    blocks_o, _ = odg.assemble(p, ingr, alpha)
    dV = sols[0]["dV"]
    W = [sols[k]["A"] @ A_g[k].T * dV for k in range(p.n_elem)]
    worst = 0.0
    for k in range(p.n_elem):
        for s in range(p.n_stencil):
            n = int(p.neighbors[k, s])
            if n < 0:
                continue
            nk, nn = int(q.n_alb[k]), int(q.n_alb[n])
            Hg = W[k] @ blocks_g[k, s, :nk, :nn] @ W[n].T
            worst = max(worst, np.abs(Hg - blocks_o[k, s, :nk, :nn]).max())
    assert worst <= tol, worst
    ev_g = np.linalg.eigvalsh(odg.dense(p, blocks_g, q.n_alb))[:8]
    ev_o = np.linalg.eigvalsh(odg.dense(p, blocks_o, q.n_alb))[:8]
    assert np.abs(ev_g - ev_o).max() <= tol
    return worst


@pytest.mark.parametrize("stencil", [5, 9])
def test_dg_blocks_small_slab(ctx, stencil):
    from paper_2003_00407_gb300 import api
    w = make_slab(3, 2, (8, 6, 12), (16, 12, 12), 0.45, 10, 6, 5, r_cut=2.6, width=0.7, proj_width=0.7,
                  stencil=stencil)
    p, q = w.problem, w.params
    sols = {k: driver.solve_element(p, q, k, dense_route=True) for k in range(p.n_elem)}
    res = api.alb_generate(ctx, p, q, precision=0, cheb_degree=12, tol=1e-10, max_iter=400)
    blocks = api.dg_assemble(ctx, p, q, res, 20.0).cpu().numpy()
    A_g, _ = api.alb_views(p, q, res)
    worst = _compare(w, blocks, [a.cpu().numpy() for a in A_g], sols, 20.0)
    print("max block error", worst)


def test_dg_blocks_whole_box_2x2(ctx):
    from paper_2003_00407_gb300 import api
    w = make_slab(2, 2, (6, 6, 12), (12, 12, 12), 0.5, 10, 8, 3, stencil=STENCIL_XY9, width=0.7, proj_width=0.7,
                  r_cut=2.8, lattice=1, jitter=0.3)
    p, q = w.problem, w.params
    sols = {k: driver.solve_element(p, q, k, dense_route=True) for k in range(p.n_elem)}
    res = api.alb_generate(ctx, p, q, precision=0, cheb_degree=12, tol=1e-10, max_iter=400)
    blocks = api.dg_assemble(ctx, p, q, res, 7.0).cpu().numpy()
    A_g, _ = api.alb_views(p, q, res)
    _compare(w, blocks, [a.cpu().numpy() for a in A_g], sols, 7.0)
