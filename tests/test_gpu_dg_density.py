"""The DG solution on the GPU (the steps after H^DG): electron density from the diagonal density-matrix
blocks (Eq. density, Eq. densitymatrix), the band energy (Eq. DGvar on the DG eigenpairs) and the
Hellmann-Feynman gradient at fixed ALBs (Eq. hfforce for the wells and projectors of this model), against
the oracle (oracle/dg_solve.py: dg_density, dg_band_gradient, the latter pinned by central differences).

Whole-box 2x2 elements (every Q is the whole box, 9-block stencil): GPU ALBs, blocks, DG eigensolve and
density against the oracle's dense-route ALBs, blocks and dense eigensolve.  The quantities compared are
basis invariant.  The c2 slab is compared against its stored oracle values in test_gpu_dg_contract.py.
"""
import numpy as np
import pytest

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


def global_rho(p, rho_elems):
    """Per-element densities on E_k (oracle layout) placed on the domain grid."""
    rho = np.zeros(p.v_extra.size)
    for k in range(p.n_elem):
        dom = int(p.elem_dom[k])
        n = p.dom_n[dom]
        En = p.elem_En[k]
        gE = [np.mod(p.elem_E0[k][a] + np.arange(int(En[a])), n[a]) for a in range(3)]
        flat = (gE[2][:, None, None] * n[1] + gE[1][None, :, None]) * n[0] + gE[0][None, None, :]
        rho[int(p.dom_voff[dom]) + flat.ravel()] += rho_elems[k]
    return rho


def test_whole_box_density_energy_and_forces(ctx):
    from paper_2003_00407_gb300 import api
    from oracle import driver, dg, dg_solve
    from workloads.configs import make_slab
    from workloads.problem import STENCIL_XY9
    w = make_slab(2, 2, (6, 6, 12), (12, 12, 12), 0.5, 8, 6, 3, stencil=STENCIL_XY9, width=0.7, proj_width=0.7,
                  r_cut=2.8, lattice=1, jitter=0.3)
    p, q = w.problem, w.params
    alpha, n, n_el, kT = 20.0, 12, 6.0, 0.02
    sols = {k: driver.solve_element(p, q, k, dense_route=True) for k in range(p.n_elem)}
    blocks_o, _ = driver.dg_assemble(p, sols, alpha)
    eps, V = np.linalg.eigh(dg.dense(p, blocks_o, q.n_alb))
    rho_o, mu_o, E_o = dg_solve.dg_density(p, sols, q.n_alb, eps[:n], V[:, :n].T, n_el, kT)
    _, _, gR_o = dg_solve.dg_band_gradient(p, sols, q.n_alb, eps[:n], V[:, :n].T, n_el, kT)
    rho_o = global_rho(p, rho_o)
    res = api.alb_generate(ctx, p, q, precision=0, cheb_degree=12, tol=1e-11, max_iter=400)
    blocks = api.dg_assemble(ctx, p, q, res, alpha)
    ev, rs, vec, _ = api.dg_eigensolve(ctx, p, q, blocks, n, 16, cheb_degree=20, tol=1e-11, max_iter=500)
    rho, E, mu, gR = api.dg_density(ctx, p, q, res, ev[:n], vec[:n], n, n_el, kT)
    rho, gR = rho.cpu().numpy(), gR.cpu().numpy()
    dV = float(np.prod(p.dom_h[0]))
    d_rho = np.abs(rho - rho_o).max() / rho_o.max()
    d_R = np.abs(gR - gR_o).max() / np.abs(gR_o).max()
    print(f"whole box: band energy {E:.10f} vs {E_o:.10f}, mu {mu:.6f} vs {mu_o:.6f}, rho rel {d_rho:.2e}, "
          f"grad_R rel {d_R:.2e}, charge {rho.sum() * dV:.12f}")
    assert abs(rho.sum() * dV - n_el) <= 1e-9
    assert abs(E - E_o) <= 1e-8 and abs(mu - mu_o) <= 1e-6
    assert d_rho <= 1e-7
    assert d_R <= 1e-6


def test_occupied_top_state_is_reported(ctx):
    from paper_2003_00407_gb300 import api
    from workloads.configs import make_slab
    from workloads.problem import STENCIL_XY9
    w = make_slab(2, 2, (6, 6, 12), (12, 12, 12), 0.5, 8, 6, 3, stencil=STENCIL_XY9, width=0.7, proj_width=0.7,
                  r_cut=2.8, lattice=1, jitter=0.3)
    p, q = w.problem, w.params
    res = api.alb_generate(ctx, p, q, precision=0, cheb_degree=12, tol=1e-10, max_iter=400)
    blocks = api.dg_assemble(ctx, p, q, res, 20.0)
    ev, rs, vec, _ = api.dg_eigensolve(ctx, p, q, blocks, 4, 8, cheb_degree=20, tol=1e-10, max_iter=500)
    with pytest.raises(api.DgdftError) as e:
        api.dg_density(ctx, p, q, res, ev[:4], vec[:4], 4, 8.0, 0.02)     # 8 electrons in 4 states
    assert "BAD_INPUT" in str(e.value)
