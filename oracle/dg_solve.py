"""Eigenpairs of the assembled DG Hamiltonian (Eq. DGEigenvalue) by Chebyshev-filtered subspace
iteration (Alg. CheFSI, which the paper applies to H^DG) -- TEST INFRASTRUCTURE (see the package
header).

The DG basis (the ALBs of all elements) is orthonormal, so the problem is the standard symmetric one
H^DG c = eps c with the Euclidean inner product.  H^DG is never formed: it is applied block by block
from the stencil blocks of ``dg.assemble`` (block (k, s) couples the test ALBs of element k with the
trial ALBs of element neighbors[k][s]), which is the same sum ``dg.dense`` forms.
"""
from __future__ import annotations

import numpy as np

from . import chefsi as cf


class DGOperator:
    """H^DG applied to rows of X [n_vec, N_b] (N_b = sum of n_alb over elements)."""

    def __init__(self, prob, blocks, n_alb):
        self.prob = prob
        self.blocks = blocks
        self.n_alb = np.asarray(n_alb, dtype=np.int64)
        self.off = np.concatenate([[0], np.cumsum(self.n_alb)])
        self.N = int(self.off[-1])
        self.dV = 1.0

    def apply(self, X):
        X = np.atleast_2d(X)
        Y = np.zeros_like(X, dtype=np.float64)
        p, off, na = self.prob, self.off, self.n_alb
        for k in range(p.n_elem):
            for s in range(p.n_stencil):
                kp = int(p.neighbors[k, s])
                if kp < 0:
                    continue
                B = self.blocks[k, s, :na[k], :na[kp]]
                Y[:, off[k]:off[k + 1]] += X[:, off[kp]:off[kp + 1]] @ B.T
        return Y


def dg_eigenpairs(prob, blocks, n_alb, n_states, n_blk, degree, tol, max_iter, seed):
    """Lowest n_states eigenpairs of H^DG (CheFSI from a SplitMix64 start, element index 0).

    Returns the CheFSI dict: theta [n_blk], X [n_blk, N_b] (rows orthonormal), resid, iters, converged."""
    op = DGOperator(prob, blocks, n_alb)
    X0 = cf.random_block(seed, 0, n_blk, op.N)
    return cf.chefsi(op, n_states, n_blk, degree, tol, max_iter, X0)


def dg_density(prob, sols, n_alb, eps, C, n_electrons, kT):
    """Electron density of the DG solution (Sec. II.A: rho = sum_i 2 f_i |psi_i|^2 with
    psi_i = sum_{k,a} c_{i,ka} phi_{k,a}, each ALB phi_{k,a} supported on E_k).

    eps [n] and C [n, N_b] (rows orthonormal) are DG eigenpairs; f_i is Fermi-Dirac at kT with mu fixed by
    sum_i 2 f_i = n_electrons.  Returns (rho per element [M] arrays on E_k, mu, band energy sum 2 f eps)."""
    from .grad import fermi, fermi_level
    eps = np.asarray(eps, dtype=np.float64)
    mu = fermi_level(eps, float(n_electrons), kT)
    f = fermi(eps, mu, kT)
    off = np.concatenate([[0], np.cumsum(np.asarray(n_alb, dtype=np.int64))])
    rho = []
    for k in range(prob.n_elem):
        A = sols[k]["A"]                                  # [n_alb_k, N_E] on E_k
        psi = C[:, off[k]:off[k + 1]] @ A                 # [n, N_E]
        rho.append((2.0 * f[:, None] * psi * psi).sum(axis=0))
    return rho, mu, float((2.0 * f * eps).sum())
