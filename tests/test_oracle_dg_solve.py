"""Pins of the global DG eigensolve (Eq. DGEigenvalue by Alg. CheFSI on H^DG)."""
import numpy as np

from oracle import dg, dg_solve
from test_oracle_dg import _whole_box_2x2, _sols_dense, _ingredients


def _case():
    w = _whole_box_2x2(8, 6)
    sols = _sols_dense(w)
    blocks, _ = dg.assemble(w.problem, _ingredients(w, sols), 20.0)
    return w, blocks


def test_blockwise_application_is_the_assembled_matrix():
    w, blocks = _case()
    p, n_alb = w.problem, w.params.n_alb
    H = dg.dense(p, blocks, n_alb)
    op = dg_solve.DGOperator(p, blocks, n_alb)
    X = np.random.default_rng(4).normal(size=(5, op.N))
    np.testing.assert_allclose(op.apply(X), X @ H.T, atol=1e-12)
    np.testing.assert_allclose(H, H.T, atol=1e-12)


def test_chefsi_on_hdg_matches_dense_eigensolve():
    w, blocks = _case()
    p, n_alb = w.problem, w.params.n_alb
    ref = np.linalg.eigvalsh(dg.dense(p, blocks, n_alb))
    r = dg_solve.dg_eigenpairs(p, blocks, n_alb, n_states=6, n_blk=10, degree=12, tol=1e-10, max_iter=300,
                               seed=11)
    assert r["converged"]
    np.testing.assert_allclose(r["theta"][:6], ref[:6], atol=1e-9)
    X = r["X"][:6]
    np.testing.assert_allclose(X @ X.T, np.eye(6), atol=1e-10)
    H = dg.dense(p, blocks, n_alb)
    R = X @ H.T - r["theta"][:6, None] * X
    assert np.sqrt((R * R).sum(axis=1)).max() <= 1e-10


def test_density_integrates_to_the_electron_count_and_matches_the_density_matrix():
    w, blocks = _case()
    p, n_alb = w.problem, w.params.n_alb
    sols = _sols_dense(w)
    H = dg.dense(p, blocks, n_alb)
    eps, V = np.linalg.eigh(H)
    C = V[:, :10].T
    n_el, kT = 6.0, 0.05
    rho, mu, e_band = dg_solve.dg_density(p, sols, n_alb, eps[:10], C, n_el, kT)
    dV = sols[0]["dV"]
    # the ALBs are dV-orthonormal on each E_k and the rows of C orthonormal: integral = sum 2 f = N_e
    assert abs(sum(r.sum() for r in rho) * dV - n_el) <= 1e-9
    assert all(np.all(r >= -1e-14) for r in rho)
    # band energy = tr(H D) with the DG density matrix D = sum_i 2 f_i c_i c_i^T
    from oracle.grad import fermi
    f = fermi(eps[:10], mu, kT)
    D = (C.T * (2.0 * f)) @ C
    assert abs(e_band - np.trace(H @ D)) <= 1e-10 * max(1.0, abs(e_band))


def _band_energy_fixed_albs(w, sols, n_states, n_el, kT, alpha=20.0):
    """E_DG of the lowest n_states DG eigenpairs with the ALBs of `sols` held fixed (the problem's atoms
    may have moved): H^DG re-assembled from the same ALBs, eigh, Fermi-smeared band energy."""
    from oracle.grad import band_energy_weights
    p = w.problem
    ingr = [dg.element_ingredients(p, k, sols[k]["X"][:sols[k]["n_eig"]], sols[k]["C"], sols[k]["A"])
            for k in range(p.n_elem)]
    blocks, _ = dg.assemble(p, ingr, alpha)
    eps = np.linalg.eigvalsh(dg.dense(p, blocks, w.params.n_alb))[:n_states]
    return band_energy_weights(eps, n_el, kT)[0]


def test_dg_band_gradient_matches_central_differences():
    """dE_DG/dR at fixed ALBs (the DG Hellmann-Feynman force, Eq. hfforce) against central differences of
    the re-assembled, re-diagonalised DG band energy (step 1e-4 bohr, error O(1e-8))."""
    import copy
    w, blocks = _case()
    p, n_alb = w.problem, w.params.n_alb
    sols = _sols_dense(w)
    H = dg.dense(p, blocks, n_alb)
    eps, V = np.linalg.eigh(H)
    n, n_el, kT = 12, 6.0, 0.02
    E, mu, gR = dg_solve.dg_band_gradient(p, sols, n_alb, eps[:n], V[:, :n].T, n_el, kT)
    assert abs(E - _band_energy_fixed_albs(w, sols, n, n_el, kT)) <= 1e-12
    step = 1e-4
    worst = 0.0
    for a in range(p.n_atoms):
        for ax in range(3):
            Es = []
            for sgn in (1, -1):
                w2 = copy.deepcopy(w)
                w2.problem.atom_pos[a, ax] += sgn * step
                Es.append(_band_energy_fixed_albs(w2, sols, n, n_el, kT))
            fd = (Es[0] - Es[1]) / (2 * step)
            worst = max(worst, abs(fd - gR[a, ax]))
    assert worst <= 1e-6 * max(1.0, np.abs(gR).max()), (worst, np.abs(gR).max())
    assert np.abs(gR).max() > 1e-3        # the test moves something
