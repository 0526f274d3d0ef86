"""Chebyshev-filtered subspace iteration on one extended element (Alg. CheFSI).

The paper applies CheFSI to the DG Hamiltonian; here it solves the local
plane-wave problem of Eq. LocalKS (its LOBPCG default is replaced by CheFSI).
Steps per iteration, in the algorithm's order:

1. bounds: b_up from a few Lanczos steps (largest Ritz value of the Lanczos
   tridiagonal plus the norm of the last residual); b_low = the largest Ritz
   value of the current block; a0 = the smallest (used to scale the filter);
2. filter  Y = p_m(H) X  with [b_low, b_up] mapped to [-1, 1], by the scaled
   three-term Chebyshev recurrence (Zhou, Saad, Tiago, Chelikowsky 2006);
3. Cholesky-QR: S = Y^T Y dV = U^T U, Y_hat = Y U^{-1} (done twice, CholQR2;
   the paper's garbled "Y_hat U = Y_tilde" read as this);
4. Rayleigh-Ritz: H_hat = Y_hat^T H Y_hat dV, H_hat V = V D;
5. rotation X = Y_hat V;  6. X is the next block.

Convergence: every one of the n_eig lowest Ritz pairs has residual
||H x - lambda x|| (dV norm) <= tol, or max_iter filter passes were made.
Before the first filter pass the random start is orthonormalised and one
Rayleigh-Ritz step gives the first bounds.

The random start is SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a
counter-based generator: value(c) is the (c+1)-th output of SplitMix64
seeded with `seed`, with counter c = elem * 2^40 + vec * 2^24 + point; the top
53 bits give u in [0, 1) and the entry is 2u - 1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_value(seed, counter):
    """(counter+1)-th SplitMix64 output for state `seed` (vectorised, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        z = np.uint64(seed) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def random_block(seed, elem, n_vec, N):
    """Random start [n_vec, N] with entries uniform in [-1, 1)."""
    with np.errstate(over="ignore"):
        base = np.uint64(elem) << np.uint64(40)
        v = np.arange(n_vec, dtype=np.uint64)[:, None] << np.uint64(24)
        p = np.arange(N, dtype=np.uint64)[None, :]
        z = splitmix64_value(seed, base + v + p)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def lanczos_upper_bound(op, v0, steps):
    """Upper bound of the spectrum: max Ritz value of the k-step Lanczos tridiagonal + |f_k|."""
    v = v0 / np.linalg.norm(v0)
    f = op.apply(v[None, :])[0]
    a = float(v @ f)
    f = f - a * v
    alphas, betas = [a], []
    for _ in range(1, steps):
        b = float(np.linalg.norm(f))
        if b == 0.0:
            break
        v_old, v = v, f / b
        f = op.apply(v[None, :])[0] - b * v_old
        a = float(v @ f)
        f = f - a * v
        alphas.append(a)
        betas.append(b)
    T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
    return float(np.linalg.eigvalsh(T)[-1] + np.linalg.norm(f))


def cholqr(Y, dV):
    """One Cholesky-QR pass on a row block: returns Y_hat with Y_hat Y_hat^T dV = I."""
    S = (Y @ Y.T) * dV
    S = 0.5 * (S + S.T)
    U = np.linalg.cholesky(S).T            # S = U^T U, U upper triangular
    return sla.solve_triangular(U, Y, trans="T", lower=False)  # rows of (Y_col U^{-1})^T


def cholqr2(Y, dV):
    return cholqr(cholqr(Y, dV), dV)


def rayleigh_ritz(op, Y):
    """Rayleigh-Ritz on an orthonormal row block: (theta, X, HX, resid)."""
    HY = op.apply(Y)
    Hh = (Y @ HY.T) * op.dV
    Hh = 0.5 * (Hh + Hh.T)
    theta, V = np.linalg.eigh(Hh)
    X = V.T @ Y
    HX = V.T @ HY
    R = HX - theta[:, None] * X
    resid = np.sqrt((R * R).sum(axis=1) * op.dV)
    return theta, X, HX, resid


def chebyshev_filter(op, X, m, b_low, b_up, a0):
    """Y = p_m(H) X: degree-m Chebyshev filter damping [b_low, b_up], scaled at a0."""
    e = 0.5 * (b_up - b_low)
    c = 0.5 * (b_up + b_low)
    sigma = e / (a0 - c)
    sigma1 = sigma
    Y = (op.apply(X) - c * X) * (sigma1 / e)
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (2.0 / sigma1 - sigma)
        Y_new = (op.apply(Y) - c * Y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * X
        X, Y = Y, Y_new
        sigma = sigma_new
    return Y


def chefsi(op, n_eig, n_blk, degree, tol, max_iter, X0, lanczos_steps=10):
    """Lowest n_eig eigenpairs of op by CheFSI.

    Returns dict(theta [n_blk], X [n_blk, N], resid [n_blk], iters, converged,
    b_up, history).  Rows of X are dV-orthonormal.
    """
    X = cholqr2(np.array(X0, dtype=np.float64), op.dV)
    b_up = lanczos_upper_bound(op, X0[0].astype(np.float64), lanczos_steps)
    theta, X, HX, resid = rayleigh_ritz(op, X)
    hist = [float(resid[:n_eig].max())]
    it = 0
    converged = bool(resid[:n_eig].max() <= tol)
    while not converged and it < max_iter:
        a0, b_low = theta[0], theta[-1]
        Y = chebyshev_filter(op, X, degree, b_low, b_up, a0)
        Y = cholqr2(Y, op.dV)
        theta, X, HX, resid = rayleigh_ritz(op, Y)
        it += 1
        hist.append(float(resid[:n_eig].max()))
        converged = bool(resid[:n_eig].max() <= tol)
    return dict(theta=theta, X=X, resid=resid, iters=it, converged=converged, b_up=b_up,
                history=hist)
