"""Pins of the ALB restriction and SVD truncation."""
import numpy as np

from oracle import alb, driver
from workloads import make_config
from helpers import subspace_sine


def test_restrict_indices():
    Qn, eo, En = (6, 5, 4), (1, 2, 0), (3, 2, 4)
    X = np.arange(2 * 120, dtype=float).reshape(2, 120)
    R = alb.restrict(X, Qn, eo, En)
    z, y, x = np.meshgrid(np.arange(4), np.arange(2, 4), np.arange(1, 4), indexing="ij")
    np.testing.assert_array_equal(R[1], X[1][(z * 5 + y) * 6 + x].ravel())


def test_svd_and_gram_routes_agree():
    rng = np.random.default_rng(0)
    Phi = rng.normal(size=(10, 300))
    dV = 0.2
    A1, C1, s1 = alb.svd_truncate(Phi, 6, dV)
    A2, C2, s2 = alb.gram_truncate(Phi, 6, dV)
    np.testing.assert_allclose(s1, s2, rtol=1e-10)
    np.testing.assert_allclose(A1, A2, atol=1e-9)
    np.testing.assert_allclose(A1, C1.T @ Phi, atol=1e-10)
    np.testing.assert_allclose(A1 @ A1.T * dV, np.eye(6), atol=1e-12)
    # singular values by numpy's dense SVD of the scaled block
    np.testing.assert_allclose(s1, np.linalg.svd(Phi * np.sqrt(dV), compute_uv=False), rtol=1e-12)


def test_alb_config1_properties():
    w = make_config(1)
    s = driver.solve_element(w.problem, w.params, 0, dense_route=True)
    assert np.all(s["sing"] <= 1.0 + 1e-12)             # restriction of orthonormal vectors
    A = s["A"]
    np.testing.assert_allclose(A @ A.T * s["dV"], np.eye(8), atol=1e-12)
    # ALB span = top-8 left singular subspace of the restricted block
    from oracle import local_operator as lo
    Phi_E = alb.restrict(s["X"][:16], w.problem.elem_Qn[0], lo.e_offset_in_q(w.problem, 0),
                         w.problem.elem_En[0])
    U, sv, Wt = np.linalg.svd(Phi_E.T, full_matrices=False)
    assert subspace_sine(U[:, :8].T / np.sqrt(s["dV"]), A, s["dV"]) < 1e-10
