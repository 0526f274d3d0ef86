"""Fermi-smeared band energy of the local problems and its exact gradient.

The paper's forces are Hellmann-Feynman forces (Eq. hfforce).  The local
analogue computed here is, per element k,

    E_k = sum_{j <= n_eig} 2 f_j lambda_j,   f_j = 1 / (1 + exp((lambda_j - mu_k) / kT)),

with the spin factor 2 (closed shell) and mu_k fixed by sum_j 2 f_j = N_el,k
(bisection).  For the discrete operator, Hellmann-Feynman is exact:

    dE_k/dtheta = sum_j w_j <phi_j, dH/dtheta phi_j>,
    w_j = 2 [f_j + f'_j (lambda_j - mu_bar)],  mu_bar = sum lambda f' / sum f',

where the mu_bar term comes from the electron-count constraint.  With H =
T + diag(V_Q) + sum gamma b b^T dV and V_Q the restriction of the global V:

    dE/dV(g)  = sum_k sum_j w_j sum_{q in Q_k -> g} phi_j(q)^2 dV
    dE/dR_I   = sum_k sum_j w_j [ sum_q phi_j(q)^2 dV_I(q)/dR_I dV
                                  + 2 sum_l gamma_l <phi_j, b_l> <phi_j, db_l/dR_I> ].
"""
from __future__ import annotations

import numpy as np

from .local_operator import q_global_indices, displacements, projector_norms, taper


def fermi(lam, mu, kT):
    x = np.clip((lam - mu) / kT, -700.0, 700.0)
    return 1.0 / (1.0 + np.exp(x))


def fermi_level(lam, n_el, kT, iters=200):
    """mu with sum_j 2 f(lambda_j) = n_el, by bisection."""
    lo = float(lam.min()) - 50.0 * kT - 1.0
    hi = float(lam.max()) + 50.0 * kT + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if 2.0 * fermi(lam, mid, kT).sum() > n_el:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def band_energy_weights(lam, n_el, kT):
    """(E, mu, w) for eigenvalues lam of one element."""
    mu = fermi_level(lam, n_el, kT)
    f = fermi(lam, mu, kT)
    fp = -f * (1.0 - f) / kT
    E = float((2.0 * f * lam).sum())
    sfp = fp.sum()
    mu_bar = float((lam * fp).sum() / sfp) if sfp != 0.0 else 0.0
    w = 2.0 * (f + fp * (lam - mu_bar))
    return E, mu, w, f


def _dgauss_taper(DX, DY, DZ, sigma, r_cut):
    """g = exp(-d^2/2 sigma^2) tau(d/r_cut) and its gradient w.r.t. the displacement d."""
    d2 = DX * DX + DY * DY + DZ * DZ
    s2 = d2 / (r_cut * r_cut)
    inside = s2 < 1.0
    ga = np.exp(-d2 / (2.0 * sigma * sigma))
    one = np.where(inside, 1.0 - s2, 0.0)
    g = ga * one ** 3
    common = ga * (-(one ** 3) / (sigma * sigma) - 6.0 * one ** 2 / (r_cut * r_cut))
    return g, (common * DX, common * DY, common * DZ)


def element_gradient(prob, k, lam, Phi, n_el, kT, grad_v, grad_R):
    """Accumulate element k's contributions into grad_v (per-domain flat) and grad_R; returns E_k."""
    dom = int(prob.elem_dom[k])
    h = prob.dom_h[dom]
    dV = float(np.prod(h))
    E, mu, w, f = band_energy_weights(lam, n_el, kT)
    if f[-1] >= 1e-12:
        raise ValueError("top eigenvalue is occupied (f >= 1e-12): enlarge n_eig")
    rho = (w[:, None] * Phi * Phi).sum(0) * dV          # sum_j w_j phi_j^2 dV on Q
    Qn = prob.elem_Qn[k]
    rho3 = rho.reshape(int(Qn[2]), int(Qn[1]), int(Qn[0]))
    gx, gy, gz = q_global_indices(prob, k)
    n = prob.dom_n[dom]
    flat = (gz[:, None, None] * n[1] + gy[None, :, None]) * n[0] + gx[None, None, :]
    np.add.at(grad_v, int(prob.dom_voff[dom]) + flat.ravel(), rho3.ravel())
    for a in range(prob.n_atoms):
        if int(prob.atom_dom[a]) != dom:
            continue
        DX, DY, DZ = displacements(prob, dom, gx, gy, gz, prob.atom_pos[a])
        if not np.any(taper(np.sqrt(DX * DX + DY * DY + DZ * DZ) / prob.r_cut) > 0):
            continue
        # local wells: V_I = -D g(d), dV_I/dR = +D dg/dd
        _, dg = _dgauss_taper(DX, DY, DZ, prob.well_width[a], prob.r_cut)
        for ax in range(3):
            grad_R[a, ax] += prob.well_depth[a] * float((rho3 * dg[ax]).sum())
        if prob.n_proj_per_atom == 0:
            continue
        sig = prob.proj_width[a]
        g, dgp = _dgauss_taper(DX, DY, DZ, sig, prob.r_cut)
        ns, np_ = projector_norms(sig)
        disp = (DX, DY, DZ)
        b = [ns * g] + ([np_ * disp[0] * g, np_ * disp[1] * g, np_ * disp[2] * g]
                        if prob.n_proj_per_atom == 4 else [])
        for l in range(prob.n_proj_per_atom):
            pb = Phi @ b[l].ravel() * dV                      # <phi_j, b_l>
            for ax in range(3):
                if l == 0:
                    db = -ns * dgp[ax]
                else:
                    beta = l - 1
                    db = -np_ * ((g if beta == ax else 0.0) + disp[beta] * dgp[ax])
                pdb = Phi @ np.asarray(db).ravel() * dV        # <phi_j, db_l/dR_ax>
                grad_R[a, ax] += float((w * 2.0 * prob.proj_gamma[a, l] * pb * pdb).sum())
    return E
