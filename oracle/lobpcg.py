"""LOBPCG with the Teter preconditioner on one extended element (Alg. LOBPCG, Eqs. 3-5) -- TEST
INFRASTRUCTURE (see the package header).

The paper's default plane-wave eigensolver for small local problems.  Per iteration, in the algorithm's
order:

1. W = T R with R = H X - X (X^T H X) dV (Eq. 3), T the Teter preconditioner (below);
2. trial subspace S = [X, W, P] (P absent in the first iteration); the rows of W and P are scaled to unit
   norm first, which leaves the subspace unchanged and keeps S^T S well conditioned as R -> 0;
3. the projected generalized problem S^T H S C = S^T S C Lambda (Eq. 5), lowest n_blk pairs;
4. P = W C_W + P C_P (the conjugate direction), X = X C_X + P (Eq. 4).

Teter preconditioner (Teter, Payne and Allan, Phys. Rev. B 40, 12255 (1989)): in the plane-wave basis it
multiplies the coefficient of G in the residual of band i by

    K(x) = (27 + 18 x + 12 x^2 + 8 x^3) / (27 + 18 x + 12 x^2 + 8 x^3 + 16 x^4),  x = (|G|^2 / 2) / E_i,

with E_i = <x_i, T x_i> dV the kinetic energy of band i.  K(0) = 1, K decreases monotonically and
K(x) -> 1 / (2 x) for large x: in the tail it falls like the inverse kinetic energy, which is what a
preconditioner of H - theta needs.

Convergence: as in oracle/chefsi.py -- every one of the n_eig lowest Ritz pairs has residual
||H x - theta x|| (dV norm) <= tol, or max_iter iterations were made.  The result has the same plain
definition as the CheFSI route: the lowest eigenpairs of H.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .chefsi import cholqr2


def teter_factor(x):
    """K(x) of the Teter preconditioner for x >= 0."""
    x = np.asarray(x, dtype=np.float64)
    num = 27.0 + 18.0 * x + 12.0 * x * x + 8.0 * x ** 3
    return num / (num + 16.0 * x ** 4)


def kinetic_energy(op, X):
    """<x_i, T x_i> dV for the rows of X."""
    return (X * op.kinetic(X)).sum(axis=1) * op.dV


def teter_precondition(op, R, ekin):
    """W = T R: per row i, the spectrum of R_i scaled by K(|G|^2/2 / ekin_i)."""
    nv = R.shape[0]
    F = np.fft.rfftn(R.reshape((nv,) + op.shape), axes=(1, 2, 3))
    x = op.K[None] / np.maximum(ekin, 1e-300)[:, None, None, None]
    return np.fft.irfftn(F * teter_factor(x), s=op.shape, axes=(1, 2, 3)).reshape(nv, op.N)


def lobpcg(op, n_eig, n_blk, tol, max_iter, X0):
    """Lowest n_eig eigenpairs of op (block n_blk).  Returns the dict of oracle/chefsi.chefsi."""
    dV = op.dV
    X = cholqr2(np.array(X0, dtype=np.float64), dV)
    HX = op.apply(X)
    Hh = (X @ HX.T) * dV
    theta, V = np.linalg.eigh(0.5 * (Hh + Hh.T))
    X, HX = V.T @ X, V.T @ HX
    P = HP = None
    hist = []
    it = 0
    while True:
        R = HX - theta[:, None] * X
        resid = np.sqrt((R * R).sum(axis=1) * dV)
        hist.append(float(resid[:n_eig].max()))
        if resid[:n_eig].max() <= tol or it >= max_iter:
            break
        W = teter_precondition(op, R, kinetic_energy(op, X))
        W = W / np.sqrt((W * W).sum(axis=1) * dV)[:, None]   # unit rows: same span, better-conditioned S^T S
        HW = op.apply(W)
        parts = [X, W] + ([P] if P is not None else [])
        hparts = [HX, HW] + ([HP] if HP is not None else [])
        S = np.vstack(parts)
        HS = np.vstack(hparts)
        G = (S @ S.T) * dV
        A = (S @ HS.T) * dV
        G, A = 0.5 * (G + G.T), 0.5 * (A + A.T)
        lam, C = sla.eigh(A, G)                # S^T H S C = S^T S C Lambda (Eq. 5)
        C = C[:, :n_blk]
        n = n_blk
        CX, CW = C[:n], C[n:2 * n]
        CP = C[2 * n:] if P is not None else None
        P_new = CW.T @ W + (CP.T @ P if P is not None else 0.0)
        HP_new = CW.T @ HW + (CP.T @ HP if P is not None else 0.0)
        X = CX.T @ X + P_new                   # Eq. 4
        HX = CX.T @ HX + HP_new
        pn = np.sqrt((P_new * P_new).sum(axis=1) * dV)[:, None]
        P, HP = P_new / pn, HP_new / pn        # unit rows for the next trial subspace (same span)
        theta = lam[:n_blk]
        it += 1
    return dict(theta=theta, X=X, resid=resid, iters=it, converged=bool(resid[:n_eig].max() <= tol),
                history=hist)
