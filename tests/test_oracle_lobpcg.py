"""Pins of the LOBPCG + Teter oracle (Alg. LOBPCG, Eqs. 3-5): the preconditioner polynomial against its
defining properties, and the converged eigenpairs against the dense eigensolve (their plain definition)."""
import numpy as np

from oracle import chefsi as cf, local_operator as lo, lobpcg as lp
from workloads import make_config
from workloads.configs import make_slab


def test_teter_factor_properties():
    x = np.linspace(0.0, 50.0, 2001)
    K = lp.teter_factor(x)
    assert K[0] == 1.0
    assert np.all(np.diff(K) < 0)                                  # monotone
    big = np.array([1e3, 1e4, 1e5])
    np.testing.assert_allclose(lp.teter_factor(big) * 2 * big, 1.0, rtol=2e-3)   # tail 1/(2x)
    # the polynomial written out at x = 1: 65 / 81
    assert abs(lp.teter_factor(1.0) - 65.0 / 81.0) < 1e-15


def test_preconditioner_is_a_symmetric_positive_spectral_multiplier():
    w = make_config(1)
    op = lo.LocalOperator(w.problem, 0)
    rng = np.random.default_rng(0)
    A, B = rng.normal(size=(2, op.N)), rng.normal(size=(2, op.N))
    e = np.array([0.7, 0.7])
    TA, TB = lp.teter_precondition(op, A, e), lp.teter_precondition(op, B, e)
    assert abs((A * TB).sum() - (TA * B).sum()) <= 1e-10 * np.abs(A * TB).sum()
    assert (A * TA).sum(axis=1).min() > 0
    # the constant mode (G = 0) is left unchanged
    one = np.ones((1, op.N))
    np.testing.assert_allclose(lp.teter_precondition(op, one, np.array([1.3])), one, atol=1e-12)


def test_lobpcg_matches_the_dense_eigensolve_with_wells():
    w = make_config(1)
    p, q = w.problem, w.params
    op = lo.LocalOperator(p, 0)
    ref = np.linalg.eigvalsh(lo.dense_matrix(op))
    X0 = cf.random_block(q.seed, 0, 24, op.N)
    r = lp.lobpcg(op, 16, 24, 1e-9, 400, X0)
    assert r["converged"], r["history"][-5:]
    np.testing.assert_allclose(r["theta"][:16], ref[:16], atol=1e-9)
    X = r["X"][:16]
    np.testing.assert_allclose(X @ X.T * op.dV, np.eye(16), atol=1e-10)
    R = op.apply(X) - r["theta"][:16, None] * X
    assert np.sqrt((R * R).sum(axis=1) * op.dV).max() <= 1e-9


def test_lobpcg_matches_chefsi_with_projectors():
    w = make_slab(3, 2, (8, 6, 12), (16, 12, 12), 0.45, 10, 6, 5, r_cut=2.6, width=0.7, proj_width=0.7)
    p, q = w.problem, w.params
    op = lo.LocalOperator(p, 2)
    X0 = cf.random_block(q.seed, 2, int(q.n_blk[2]), op.N)
    r = lp.lobpcg(op, 10, int(q.n_blk[2]), 1e-9, 400, X0)
    ref = cf.chefsi(op, 10, int(q.n_blk[2]), 12, 1e-10, 400, X0)
    assert r["converged"] and ref["converged"]
    np.testing.assert_allclose(r["theta"][:10], ref["theta"][:10], atol=1e-9)
