"""Pins of the band-energy gradient (Hellmann-Feynman analogue of Eq. hfforce): finite differences."""
import copy
import numpy as np
import pytest

from oracle import driver, grad as gr
from workloads.configs import make_slab


def _case():
    # 2x1 elements of 6x10x10 at h=0.5 (domain 6 x 5 x 5 bohr), Q 10x10x10 wrapping in x
    w = make_slab(2, 1, (6, 10, 10), (10, 10, 10), 0.5, 8, 4, 17, width=0.6, proj_width=0.6,
                  r_cut=2.4, lattice=1, jitter=0.5, zjitter=0.4)
    w.problem.v_extra = np.random.default_rng(8).normal(size=w.problem.v_extra.size) * 0.05
    w.n_electrons = np.array([4.0, 4.0])
    w.kT = 0.02
    return w


def _energy(w):
    sols = {k: driver.solve_element(w.problem, w.params, k, dense_route=True)
            for k in range(w.problem.n_elem)}
    E, gv, gR = driver.alb_grad(w.problem, sols, w.kT, w.n_electrons)
    return E.sum(), gv, gR


def test_fermi_level_counts_electrons():
    lam = np.array([-1.0, -0.5, -0.45, 0.2, 0.3])
    for n_el, kT in ((4.0, 0.01), (3.0, 0.1), (6.0, 0.05)):
        mu = gr.fermi_level(lam, n_el, kT)
        assert abs(2 * gr.fermi(lam, mu, kT).sum() - n_el) < 1e-10


def test_weights_reduce_to_occupations_when_insulating():
    lam = np.array([-1.0, -0.9, 1.0, 2.0])
    E, mu, w, f = gr.band_energy_weights(lam, 4.0, 0.001)
    np.testing.assert_allclose(w, [2, 2, 0, 0], atol=1e-12)
    assert abs(E - 2 * (-1.9)) < 1e-12


def test_gradient_wrt_atoms_matches_central_differences():
    w = _case()
    E0, gv, gR = _energy(w)
    delta = 1e-4
    for a in range(w.problem.n_atoms):
        for ax in range(3):
            wp, wm = copy.deepcopy(w), copy.deepcopy(w)
            wp.problem.atom_pos[a, ax] += delta
            wm.problem.atom_pos[a, ax] -= delta
            fd = (_energy(wp)[0] - _energy(wm)[0]) / (2 * delta)
            assert abs(fd - gR[a, ax]) < 2e-6 * max(1.0, abs(fd)), (a, ax, fd, gR[a, ax])


def test_gradient_wrt_veff_matches_central_differences():
    w = _case()
    E0, gv, gR = _energy(w)
    rng = np.random.default_rng(1)
    for _ in range(2):
        u = rng.normal(size=gv.size)
        u /= np.linalg.norm(u)
        eps = 1e-5
        wp, wm = copy.deepcopy(w), copy.deepcopy(w)
        wp.problem.v_extra = w.problem.v_extra + eps * u
        wm.problem.v_extra = w.problem.v_extra - eps * u
        fd = (_energy(wp)[0] - _energy(wm)[0]) / (2 * eps)
        assert abs(fd - gv @ u) < 1e-7 * max(1.0, abs(fd)), (fd, gv @ u)
    # total weight: sum of dE/dV over the grid = sum_j w_j (each phi_j has unit norm)
    assert abs(gv.sum() - 2 * 4.0) < 1e-6
