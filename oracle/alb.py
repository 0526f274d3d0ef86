"""Adaptive local basis: restriction to E_k and SVD truncation (Sec. II.A.1).

The J_k local eigenfunctions on Q_k are restricted to the points of E_k and
made orthonormal on E_k; they vanish outside E_k.  The paper does not name
the truncation; the reading here is the thin SVD of the restricted block:

    Phi_E sqrt(dV) = U Sigma W^T     (columns of Phi_E = restricted eigenvectors)
    ALB  A = U[:, :n_alb] / sqrt(dV)  (so A^T A dV = I on E_k)
    C    = W[:, :n_alb] Sigma^{-1}    (so A = Phi_E C)

Signs are fixed for display only: the largest-magnitude entry of each ALB is
positive (ties to the lowest index).
"""
from __future__ import annotations

import numpy as np


def restrict(X, Qn, e_off, En):
    """Rows of X on Q (x fastest) restricted to E: [n, En_z*En_y*En_x]."""
    nx, ny, nz = (int(v) for v in Qn)
    ex, ey, ez = (int(v) for v in e_off)
    mx, my, mz = (int(v) for v in En)
    X3 = np.asarray(X).reshape(X.shape[0], nz, ny, nx)
    return X3[:, ez:ez + mz, ey:ey + my, ex:ex + mx].reshape(X.shape[0], -1)


def svd_truncate(Phi_E, n_alb, dV):
    """(A [n_alb, N_E], C [n_eig, n_alb], sigma [n_eig]) from the restricted block Phi_E [n_eig, N_E]."""
    U, s, Wt = np.linalg.svd(Phi_E.T * np.sqrt(dV), full_matrices=False)
    A = U[:, :n_alb].T / np.sqrt(dV)
    C = Wt.T[:, :n_alb] / s[None, :n_alb]
    # display sign: largest |entry| of each ALB positive
    idx = np.argmax(np.abs(A), axis=1)
    sg = np.sign(A[np.arange(A.shape[0]), idx])
    sg[sg == 0] = 1.0
    return A * sg[:, None], C * sg[None, :], s


def gram_truncate(Phi_E, n_alb, dV):
    """Same truncation by the Gram route: G = Phi_E Phi_E^T dV = W Sigma^2 W^T (descending)."""
    G = Phi_E @ Phi_E.T * dV
    lam, W = np.linalg.eigh(0.5 * (G + G.T))
    order = np.argsort(lam)[::-1]
    lam, W = lam[order], W[:, order]
    s = np.sqrt(np.maximum(lam, 0.0))
    C = W[:, :n_alb] / s[None, :n_alb]
    A = C.T @ Phi_E
    idx = np.argmax(np.abs(A), axis=1)
    sg = np.sign(A[np.arange(A.shape[0]), idx])
    sg[sg == 0] = 1.0
    return A * sg[:, None], C * sg[None, :], s
