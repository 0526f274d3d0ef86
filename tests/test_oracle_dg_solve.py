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
