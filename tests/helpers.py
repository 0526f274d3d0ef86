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
