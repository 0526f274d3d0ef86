"""Comparison helpers for the tests (basis-invariant measures)."""
import numpy as np


def subspace_sine(A_ref, A, dV):
    """Sine of the largest principal angle between the row spans of A_ref and A (dV-orthonormal rows)."""
    Qr, _ = np.linalg.qr((A_ref * np.sqrt(dV)).T)
    Qa, _ = np.linalg.qr((A * np.sqrt(dV)).T)
    M = Qa - Qr @ (Qr.T @ Qa)
    return float(np.linalg.norm(M, 2))


def free_electron_levels(L, nmax):
    """Sorted 1/2 |G|^2 for a cubic box of side L over integer shells |m_i| <= nmax."""
    r = np.arange(-nmax, nmax + 1)
    MX, MY, MZ = np.meshgrid(r, r, r, indexing="ij")
    return np.sort(0.5 * (2 * np.pi / L) ** 2 * (MX ** 2 + MY ** 2 + MZ ** 2).ravel())


def oracle_element(config, k, degree, tol, max_iter, alpha=None):
    """Oracle eigenvalues, ALBs and (if alpha is given) diagonal DG block of element k of a
    configuration; runs in a worker process of the full-size tests."""
    from workloads import make_config
    from oracle import driver, dg
    w = make_config(config)
    w.params.cheb_degree = degree
    r = driver.solve_element(w.problem, w.params, k, tol=tol, max_iter=max_iter)
    out = dict(theta=r["theta"], A=r["A"], sing=r["sing"], dV=r["dV"], b_up=r["b_up"],
               resid=r["resid"], n_eig=r["n_eig"], n_alb=r["n_alb"])
    if alpha is not None:
        ik = dg.element_ingredients(w.problem, k, r["X"][:r["n_eig"]], r["C"], r["A"])
        out["dg_diag"] = dg.diagonal_block(w.problem, k, ik, alpha)
    return out
