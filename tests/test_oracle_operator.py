"""Pins of the local operator (Eq. LocalKS): closed forms, brute force, special cases."""
import os
import numpy as np
import pytest

from oracle import local_operator as lo
from oracle import chefsi as cf
from workloads import make_config
from workloads.configs import make_cube, make_slab
from helpers import free_electron_levels

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _free_op(n=16, L=10.0):
    return lo.LocalOperator.from_parts((n, n, n), (L / n,) * 3, np.zeros(n ** 3))


def test_free_electron_dense_is_closed_form():
    # dense Kronecker-sum matrix at V=0 has exactly the grid plane-wave energies
    n, L = 8, 10.0
    op = _free_op(n, L)
    ev = np.linalg.eigvalsh(lo.dense_matrix(op))
    m = np.fft.fftfreq(n) * n
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    ref = np.sort(0.5 * (2 * np.pi / L) ** 2 * (MX ** 2 + MY ** 2 + MZ ** 2).ravel())
    assert np.abs(ev - ref).max() < 1e-12


def test_free_electron_chefsi_golden_shells():
    rows = np.loadtxt(os.path.join(GOLD, "free_electron_L10.txt"))
    ref = np.concatenate([np.full(int(d), v) for v, d in rows])      # 27 levels
    np.testing.assert_allclose(ref, free_electron_levels(10.0, 1)[:27], atol=1e-14)
    op = _free_op(16, 10.0)
    n_eig = 19                                   # shell closure 1 + 6 + 12
    X0 = cf.random_block(7, 0, 24, op.N)
    r = cf.chefsi(op, n_eig, 24, 10, 1e-10, 80, X0)
    assert r["converged"]
    assert np.abs(r["theta"][:n_eig] - ref[:n_eig]).max() < 1e-10


def test_kinetic_1d_matches_trefethen_closed_form():
    # periodic spectral second-derivative matrix, Trefethen, Spectral Methods in MATLAB (Ch. 3)
    for N, L in ((16, 10.0), (24, 7.3), (48, 19.2)):
        hh = 2 * np.pi / N
        j = np.arange(N)
        with np.errstate(divide="ignore"):
            col = np.where(j == 0, -np.pi ** 2 / (3 * hh ** 2) - 1.0 / 6.0,
                           -0.5 * (-1.0) ** j / np.sin(j * hh / 2) ** 2)
        D2 = col[(j[:, None] - j[None, :]) % N]
        T = -0.5 * D2 * (2 * np.pi / L) ** 2
        assert np.abs(T - lo.kinetic_1d(N, L / N)).max() < 1e-9 * np.abs(T).max()


def test_apply_matches_dense_brute_force():
    # anisotropic, non-cubic grid with wells and projectors: FFT route == explicit matrix
    w = make_cube(11, n=12, L=7.0, n_wells=3, n_proj=4, En=6, n_eig=8, n_alb=4)
    p = w.problem
    p.dom_n[0] = (12, 10, 8); p.elem_Qn[0] = (12, 10, 8); p.elem_En[0] = (6, 6, 4)
    p.elem_E0[0] = (3, 2, 2); p.dom_h[0] = (7.0 / 12, 0.71, 0.8)
    p.v_extra = np.random.default_rng(3).normal(size=12 * 10 * 8) * 0.1
    op = lo.LocalOperator(p, 0)
    assert op.B.shape[1] == 12
    H = lo.dense_matrix(op)
    X = np.random.default_rng(0).normal(size=(5, op.N))
    np.testing.assert_allclose(op.apply(X), X @ H.T, atol=1e-10 * np.abs(H).max())
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()


def test_separable_cosine_potential_full_size():
    # V = sum_d A_d cos(2 pi x_d / L_d) on 32 x 32 x 48: 3D levels are sums of 1D levels
    n, h = (32, 32, 48), 0.4
    A = (0.8, -0.5, 1.1)
    xs = [np.arange(m) * h for m in n]
    L = [m * h for m in n]
    v1 = [A[d] * np.cos(2 * np.pi * xs[d] / L[d]) for d in range(3)]
    V = (v1[2][:, None, None] + v1[1][None, :, None] + v1[0][None, None, :]).ravel()
    op = lo.LocalOperator.from_parts(n, (h, h, h), V)
    # 1D problems from the Trefethen closed-form kinetic matrix
    e1 = []
    for d in range(3):
        N = n[d]; hh = 2 * np.pi / N; j = np.arange(N)
        with np.errstate(divide="ignore"):
            col = np.where(j == 0, -np.pi ** 2 / (3 * hh ** 2) - 1.0 / 6.0,
                           -0.5 * (-1.0) ** j / np.sin(j * hh / 2) ** 2)
        T = -0.5 * col[(j[:, None] - j[None, :]) % N] * (2 * np.pi / L[d]) ** 2
        e1.append(np.linalg.eigvalsh(T + np.diag(v1[d])))
    ref = np.sort((e1[2][:6, None, None] + e1[1][None, :6, None] + e1[0][None, None, :6]).ravel())
    n_eig = 10
    X0 = cf.random_block(1, 0, 16, op.N)
    r = cf.chefsi(op, n_eig, 16, 12, 1e-9, 80, X0)
    assert r["converged"]
    assert np.abs(r["theta"][:n_eig] - ref[:n_eig]).max() < 1e-9


def test_projector_on_exact_eigenvector_shifts_it_to_gamma():
    n, L, gamma = 10, 6.0, 1.7
    h = L / n
    dV = h ** 3
    b = np.full((n ** 3, 1), 1.0 / np.sqrt(n ** 3 * dV))      # unit-norm constant mode
    op = lo.LocalOperator.from_parts((n, n, n), (h, h, h), np.zeros(n ** 3), b, np.array([gamma]))
    ev = np.linalg.eigvalsh(lo.dense_matrix(op))
    m = np.fft.fftfreq(n) * n
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    free = np.sort(0.5 * (2 * np.pi / L) ** 2 * (MX ** 2 + MY ** 2 + MZ ** 2).ravel())
    ref = np.sort(np.concatenate([[gamma], free[1:]]))
    assert np.abs(ev - ref).max() < 1e-11
    x = b[:, 0]
    np.testing.assert_allclose(op.apply(x[None])[0], gamma * x, atol=1e-12)


def test_projector_continuum_norms():
    # without the taper (huge r_cut) on a fine grid, sum b^2 dV -> 1 for s and p
    w = make_cube(2, n=48, L=12.0, n_wells=1, n_proj=4, En=8)
    p = w.problem
    p.r_cut = 1e6
    p.atom_pos[0] = (6.0, 6.0, 6.0)
    p.proj_width[0] = 1.0
    g = np.arange(48)
    B, gam, ids = lo.projectors_on(p, 0, g, g, g)
    norms = (B * B).sum(0) * (12.0 / 48) ** 3
    np.testing.assert_allclose(norms, 1.0, atol=1e-6)
    # s and p are mutually orthogonal
    G = B.T @ B * (12.0 / 48) ** 3
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-8


def test_well_values_and_minimum_image():
    w = make_cube(2, n=20, L=10.0, n_wells=1, n_proj=0, En=8)
    p = w.problem
    p.atom_pos[0] = (0.25, 5.0, 5.0)         # near the periodic x boundary
    p.well_depth[0] = 3.0
    p.well_width[0] = 0.8
    h = 0.5
    g = np.arange(20)
    V = lo.well_potential_on(p, 0, g, g, g)
    # point (0, 5, 5) at distance 0.25 and point (19, 10, 10) at distance 0.25 through the boundary
    tau = lambda s: (1 - s * s) ** 3
    d = 0.25
    ref = -3.0 * np.exp(-d * d / (2 * 0.64)) * tau(d / 3.2)
    assert abs(V[10, 10, 0] - ref) < 1e-14
    d = 0.25 + 0.5 - 0.5 + 0.0   # x = 19*0.5 = 9.5 -> image -0.5, distance 0.75
    d = 0.75
    ref2 = -3.0 * np.exp(-d * d / (2 * 0.64)) * tau(d / 3.2)
    assert abs(V[10, 10, 19] - ref2) < 1e-14
    # outside r_cut it vanishes
    assert V[10, 10, 9] == 0.0 or abs(0.25 - 4.5) > 3.2


def test_v_local_is_restriction_of_global():
    w = make_slab(3, 2, (8, 8, 12), (16, 12, 12), 0.5, 6, 4, 5)
    p = w.problem
    p.v_extra = np.random.default_rng(2).normal(size=p.v_extra.size)
    n = p.dom_n[0]
    g = [np.arange(int(m)) for m in n]
    Vg = p.v_extra_domain(0) + lo.well_potential_on(p, 0, *g)
    for k in range(p.n_elem):
        gx, gy, gz = lo.q_global_indices(p, k)
        np.testing.assert_allclose(lo.v_local(p, k), Vg[np.ix_(gz, gy, gx)], atol=1e-13)


def test_hermitian_on_slab_element():
    w = make_slab(2, 2, (8, 8, 16), (16, 16, 16), 0.5, 6, 4, 9)
    op = lo.LocalOperator(w.problem, 3)
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=(2, op.N))
    a = x @ op.apply(y[None])[0]
    b = y @ op.apply(x[None])[0]
    assert abs(a - b) < 1e-10 * (abs(a) + 1)
