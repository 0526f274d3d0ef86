"""Pins of the CheFSI oracle (Alg. CheFSI) and its counter-based random start."""
import numpy as np
import pytest

from oracle import local_operator as lo
from oracle import chefsi as cf
from oracle import driver
from workloads import make_config
from workloads.configs import make_cube


def test_splitmix64_published_outputs():
    # first three outputs of SplitMix64 with state 0 (Vigna's splitmix64.c reference)
    v = cf.splitmix64_value(0, np.arange(3))
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_random_block_range_and_counter_layout():
    X = cf.random_block(123, 5, 3, 1000)
    assert X.shape == (3, 1000) and X.min() >= -1.0 and X.max() < 1.0
    assert abs(X.mean()) < 0.05
    # entry (elem 5, vec 2, point 7) is the value of counter 5*2^40 + 2*2^24 + 7
    z = int(cf.splitmix64_value(123, np.array([(5 << 40) + (2 << 24) + 7], dtype=np.uint64))[0])
    assert X[2, 7] == 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0


def _small_dense_op():
    w = make_cube(4, n=8, L=6.0, n_wells=3, n_proj=4, En=4)
    return lo.LocalOperator(w.problem, 0)


def test_chebyshev_filter_is_scaled_chebyshev_polynomial():
    op = _small_dense_op()
    H = lo.dense_matrix(op)
    lam, V = np.linalg.eigh(H)
    X = np.random.default_rng(1).normal(size=(4, op.N))
    m, b_low, b_up, a0 = 7, lam[40], lam[-1] + 0.5, lam[0] - 0.1
    Y = cf.chebyshev_filter(op, X, m, b_low, b_up, a0)
    e, c = 0.5 * (b_up - b_low), 0.5 * (b_up + b_low)
    T = lambda t: np.polynomial.chebyshev.chebval(t, [0] * m + [1])
    p = T((lam - c) / e) / T((a0 - c) / e)
    ref = ((X @ V) * p[None, :]) @ V.T
    assert np.abs(Y - ref).max() < 1e-10 * np.abs(ref).max()


def test_lanczos_upper_bound_bounds_spectrum():
    op = _small_dense_op()
    lam = np.linalg.eigvalsh(lo.dense_matrix(op))
    b = cf.lanczos_upper_bound(op, np.random.default_rng(0).normal(size=op.N), 10)
    assert b >= lam[-1] - 1e-9
    assert b <= lam[-1] * 1.5


def test_cholqr2_orthonormal_and_same_span():
    rng = np.random.default_rng(2)
    Y = rng.normal(size=(6, 500)) * np.array([1, 1e-3, 1, 10, 1e2, 1])[:, None]
    dV = 0.3
    Q = cf.cholqr2(Y, dV)
    assert np.abs(Q @ Q.T * dV - np.eye(6)).max() < 1e-13
    # span unchanged: Y = R^T Q for some triangular R
    R = Y @ Q.T * dV
    assert np.abs(R @ Q - Y).max() < 1e-10 * np.abs(Y).max()


def test_chefsi_matches_dense_route_config1():
    w = make_config(1)
    s = driver.solve_element(w.problem, w.params, 0, tol=1e-11, max_iter=120)
    d = driver.solve_element(w.problem, w.params, 0, dense_route=True)
    assert s["converged"]
    assert np.abs(s["theta"][:16] - d["theta"][:16]).max() < 1e-10
    assert s["resid"][:16].max() <= 1e-11
    X = s["X"]
    assert np.abs(X @ X.T * s["dV"] - np.eye(X.shape[0])).max() < 1e-12


def test_chefsi_with_projectors_matches_dense():
    w = make_cube(9, n=10, L=6.5, n_wells=3, n_proj=4, En=6, n_eig=10, n_alb=6)
    s = driver.solve_element(w.problem, w.params, 0, tol=1e-11, max_iter=150)
    d = driver.solve_element(w.problem, w.params, 0, dense_route=True)
    assert s["converged"]
    assert np.abs(s["theta"][:10] - d["theta"][:10]).max() < 1e-10


def test_rayleigh_ritz_residual_definition():
    op = _small_dense_op()
    Y = cf.cholqr2(np.random.default_rng(3).normal(size=(5, op.N)), op.dV)
    th, X, HX, r = cf.rayleigh_ritz(op, Y)
    for j in range(5):
        ref = np.sqrt(np.sum((op.apply(X[j:j + 1])[0] - th[j] * X[j]) ** 2) * op.dV)
        assert abs(r[j] - ref) < 1e-10
    assert np.all(np.diff(th) >= 0)
