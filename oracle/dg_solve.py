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


def dg_band_gradient(prob, sols, n_alb, eps, C, n_electrons, kT):
    """Fermi-smeared DG band energy and its derivative with respect to the atom positions at fixed ALBs
    (the DG form of the Hellmann-Feynman force, Eq. hfforce; the force is minus this gradient).

    E = sum_i 2 f_i eps_i over the DG eigenpairs (eps [n], rows of C [n, N_b] orthonormal), which equals
    Eq. DGvar evaluated on psi_i = sum_{k,a} C_{i,ka} phi_{k,a}.  With the ALBs held fixed, H^DG depends on
    R_I only through the local well V_I in the V_eff term and the projectors b_{I,l}, so

        dE/dR_I = sum_i w_i [ <psi_i, (dV_I/dR_I) psi_i>_T
                              + 2 sum_l gamma_l <psi_i, b_l>_T <psi_i, db_l/dR_I>_T ],
        w_i = 2 [f_i + f'_i (eps_i - mu_bar)]

    (the mu_bar term keeps the electron count fixed, as in oracle/grad.py).  The integrals over T run over
    the elements: psi_i on E_k is sum_a C_{i,ka} phi_{k,a}.  Returns (E, mu, grad_R [n_atoms, 3])."""
    from .grad import band_energy_weights, _dgauss_taper
    from .local_operator import displacements, projector_norms, taper
    eps = np.asarray(eps, dtype=np.float64)
    E, mu, w, f = band_energy_weights(eps, float(n_electrons), kT)
    off = np.concatenate([[0], np.cumsum(np.asarray(n_alb, dtype=np.int64))])
    grad_R = np.zeros((prob.n_atoms, 3))
    npa = prob.n_proj_per_atom
    pb = np.zeros((prob.n_atoms, max(npa, 1), len(eps)))
    pdb = np.zeros((prob.n_atoms, max(npa, 1), 3, len(eps)))
    for k in range(prob.n_elem):
        dom = int(prob.elem_dom[k])
        dV = float(np.prod(prob.dom_h[dom]))
        En = prob.elem_En[k]
        gE = [np.mod(prob.elem_E0[k][a] + np.arange(int(En[a])), prob.dom_n[dom][a]) for a in range(3)]
        Psi = C[:, off[k]:off[k + 1]] @ sols[k]["A"]            # [n, N_E]: psi_i on E_k
        rho_w = (w[:, None] * Psi * Psi).sum(axis=0)
        for a in range(prob.n_atoms):
            if int(prob.atom_dom[a]) != dom:
                continue
            DX, DY, DZ = displacements(prob, dom, gE[0], gE[1], gE[2], prob.atom_pos[a])
            if not np.any(taper(np.sqrt(DX * DX + DY * DY + DZ * DZ) / prob.r_cut) > 0):
                continue
            _, dgw = _dgauss_taper(DX, DY, DZ, prob.well_width[a], prob.r_cut)
            for ax in range(3):
                grad_R[a, ax] += prob.well_depth[a] * float((rho_w * dgw[ax].ravel()).sum()) * dV
            if npa == 0:
                continue
            sig = prob.proj_width[a]
            g, dgp = _dgauss_taper(DX, DY, DZ, sig, prob.r_cut)
            ns, np_ = projector_norms(sig)
            disp = (DX, DY, DZ)
            b = [ns * g] + ([np_ * disp[0] * g, np_ * disp[1] * g, np_ * disp[2] * g] if npa == 4 else [])
            for l in range(npa):
                pb[a, l] += Psi @ b[l].ravel() * dV
                for ax in range(3):
                    if l == 0:
                        db = -ns * dgp[ax]
                    else:
                        beta = l - 1
                        db = -np_ * ((g if beta == ax else 0.0) + disp[beta] * dgp[ax])
                    pdb[a, l, ax] += Psi @ np.asarray(db).ravel() * dV
    for a in range(prob.n_atoms):
        for l in range(npa):
            for ax in range(3):
                grad_R[a, ax] += float((w * 2.0 * prob.proj_gamma[a, l] * pb[a, l] * pdb[a, l, ax]).sum())
    return E, mu, grad_R
