"""Local Kohn-Sham operator on an extended element (Eq. LocalKS).

H^Q = -1/2 Laplacian + V_eff + sum_{I,l} gamma_{I,l} |b_{I,l}><b_{I,l}|

discretised on the periodic real-space grid of Q with all grid plane waves as
the basis (Sec. II.A.1: plane-wave PWDFT module; Gamma-point real
wavefunctions).  Inner products are <f, g> = sum_r f(r) g(r) dV.

Readings where the paper is silent:
* every grid mode is kept (no spherical cutoff); the kinetic multiplier keeps
  the Nyquist mode as 1/2 G^2 (even in G, so H stays real symmetric);
* V_eff on Q is the restriction of the global periodic potential: v_extra plus
  Gaussian wells V_I(r) = -D_I exp(-d^2 / 2 w_I^2) tau(d / r_cut), with d the
  minimum-image distance in the periodic domain and tau(s) = (1 - s^2)^3 for
  s < 1, else 0;
* projectors are the restriction to Q of the global periodic Gaussian-radial
  functions  b_s = N_s g,  b_p_alpha = N_p d_alpha g  with
  g = exp(-d^2 / 2 sigma^2) tau(|d| / r_cut),  N_s = (pi sigma^2)^(-3/4),
  N_p = sqrt(2) / sigma * (pi sigma^2)^(-3/4)  (continuum unit norms without
  the taper).  They are not periodised over Q.
"""
from __future__ import annotations

import numpy as np


def q_origin(prob, k):
    """Global index of Q_k's first point (may be negative; wraps periodically)."""
    return prob.elem_E0[k].astype(np.int64) - (prob.elem_Qn[k].astype(np.int64) - prob.elem_En[k]) // 2


def e_offset_in_q(prob, k):
    """Index of E_k's first point inside Q_k."""
    return (prob.elem_Qn[k].astype(np.int64) - prob.elem_En[k]) // 2


def q_global_indices(prob, k):
    """Per-axis global indices (wrapped) of Q_k's grid lines: (gx, gy, gz)."""
    d = int(prob.elem_dom[k])
    n = prob.dom_n[d].astype(np.int64)
    q0 = q_origin(prob, k)
    Qn = prob.elem_Qn[k]
    return tuple(np.mod(q0[a] + np.arange(int(Qn[a])), n[a]) for a in range(3))


def min_image(d, L):
    """Minimum-image displacement in a periodic box of length L."""
    return d - L * np.round(d / L)


def taper(s):
    """tau(s) = (1 - s^2)^3 for s < 1, else 0."""
    s = np.asarray(s, dtype=np.float64)
    return np.where(s < 1.0, (1.0 - s * s) ** 3, 0.0)


def displacements(prob, dom, gx, gy, gz, pos):
    """Minimum-image displacement r - R on the grid gz x gy x gx: arrays [nz, ny, nx] per axis."""
    h = prob.dom_h[dom]
    L = prob.dom_n[dom] * h
    dx = min_image(gx * h[0] - pos[0], L[0])
    dy = min_image(gy * h[1] - pos[1], L[1])
    dz = min_image(gz * h[2] - pos[2], L[2])
    DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
    return DX, DY, DZ


def well_potential_on(prob, dom, gx, gy, gz):
    """Sum of the Gaussian wells of domain dom on the grid lines gx, gy, gz -> [nz, ny, nx]."""
    V = np.zeros((len(gz), len(gy), len(gx)))
    for a in range(prob.n_atoms):
        if int(prob.atom_dom[a]) != dom:
            continue
        DX, DY, DZ = displacements(prob, dom, gx, gy, gz, prob.atom_pos[a])
        d2 = DX * DX + DY * DY + DZ * DZ
        w = prob.well_width[a]
        V -= prob.well_depth[a] * np.exp(-d2 / (2.0 * w * w)) * taper(np.sqrt(d2) / prob.r_cut)
    return V


def v_local(prob, k):
    """V_eff on Q_k, [Qz, Qy, Qx]: v_extra gathered with periodic wrap plus the wells."""
    dom = int(prob.elem_dom[k])
    gx, gy, gz = q_global_indices(prob, k)
    ve = prob.v_extra_domain(dom)
    V = ve[np.ix_(gz, gy, gx)].copy()
    V += well_potential_on(prob, dom, gx, gy, gz)
    return V


def projector_norms(sigma):
    """(N_s, N_p): continuum unit-norm constants of the s and p Gaussian projectors."""
    ns = (np.pi * sigma * sigma) ** (-0.75)
    return ns, np.sqrt(2.0) / sigma * ns


def projector_values(prob, a, DX, DY, DZ):
    """Projector functions of atom a at displacements (DX, DY, DZ): list of arrays, s then px, py, pz."""
    sig = prob.proj_width[a]
    d2 = DX * DX + DY * DY + DZ * DZ
    g = np.exp(-d2 / (2.0 * sig * sig)) * taper(np.sqrt(d2) / prob.r_cut)
    ns, np_ = projector_norms(sig)
    out = [ns * g]
    if prob.n_proj_per_atom == 4:
        out += [np_ * DX * g, np_ * DY * g, np_ * DZ * g]
    elif prob.n_proj_per_atom not in (0, 1):
        raise ValueError("n_proj_per_atom must be 0, 1 or 4")
    return out[:prob.n_proj_per_atom]


def projectors_on(prob, dom, gx, gy, gz):
    """All nonzero projectors of domain dom on the grid lines: (B [npts, n_p], gamma [n_p], ids [(atom, l)])."""
    cols, gam, ids = [], [], []
    if prob.n_proj_per_atom == 0:
        return np.zeros((len(gx) * len(gy) * len(gz), 0)), np.zeros(0), []
    for a in range(prob.n_atoms):
        if int(prob.atom_dom[a]) != dom:
            continue
        DX, DY, DZ = displacements(prob, dom, gx, gy, gz, prob.atom_pos[a])
        vals = projector_values(prob, a, DX, DY, DZ)
        if not np.any(vals[0] != 0.0):
            continue
        for l, v in enumerate(vals):
            cols.append(v.ravel())
            gam.append(prob.proj_gamma[a, l])
            ids.append((a, l))
    if not cols:
        return np.zeros((len(gx) * len(gy) * len(gz), 0)), np.zeros(0), []
    return np.stack(cols, axis=1), np.array(gam), ids


def kinetic_multiplier(Qn, h):
    """1/2 |G|^2 on the half spectrum [Qz, Qy, Qx//2+1] of Q (all grid modes, Nyquist kept)."""
    nx, ny, nz = (int(v) for v in Qn)
    gx = 2.0 * np.pi * np.fft.rfftfreq(nx, d=h[0])
    gy = 2.0 * np.pi * np.fft.fftfreq(ny, d=h[1])
    gz = 2.0 * np.pi * np.fft.fftfreq(nz, d=h[2])
    GZ, GY, GX = np.meshgrid(gz, gy, gx, indexing="ij")
    return 0.5 * (GX * GX + GY * GY + GZ * GZ)


class LocalOperator:
    """H^{Q_k} of element k acting on row blocks X [n_vec, N] (N = Qx*Qy*Qz, x fastest)."""

    def __init__(self, prob, k):
        self.k = k
        dom = int(prob.elem_dom[k])
        self.Qn = tuple(int(v) for v in prob.elem_Qn[k])
        self.h = prob.dom_h[dom].astype(np.float64)
        self.dV = float(np.prod(self.h))
        self.N = int(np.prod(self.Qn))
        self.shape = (self.Qn[2], self.Qn[1], self.Qn[0])
        self.V = v_local(prob, k).ravel()
        gx, gy, gz = q_global_indices(prob, k)
        self.B, self.gamma, self.proj_ids = projectors_on(prob, dom, gx, gy, gz)
        self.K = kinetic_multiplier(self.Qn, self.h)

    @classmethod
    def from_parts(cls, Qn, h, V, B=None, gamma=None):
        """Operator from explicit parts (for tests): V [N], B [N, n_p], gamma [n_p]."""
        op = cls.__new__(cls)
        op.k = -1
        op.Qn = tuple(int(v) for v in Qn)
        op.h = np.asarray(h, dtype=np.float64)
        op.dV = float(np.prod(op.h))
        op.N = int(np.prod(op.Qn))
        op.shape = (op.Qn[2], op.Qn[1], op.Qn[0])
        op.V = np.asarray(V, dtype=np.float64).ravel()
        op.B = np.zeros((op.N, 0)) if B is None else np.asarray(B, dtype=np.float64)
        op.gamma = np.zeros(0) if gamma is None else np.asarray(gamma, dtype=np.float64)
        op.proj_ids = []
        op.K = kinetic_multiplier(op.Qn, op.h)
        return op

    def kinetic(self, X):
        X = np.asarray(X, dtype=np.float64)
        nv = X.shape[0]
        F = np.fft.rfftn(X.reshape((nv,) + self.shape), axes=(1, 2, 3))
        return np.fft.irfftn(F * self.K, s=self.shape, axes=(1, 2, 3)).reshape(nv, self.N)

    def nonlocal_(self, X):
        if self.B.shape[1] == 0:
            return np.zeros_like(X)
        P = (X @ self.B) * self.dV          # <b, x>
        return (P * self.gamma) @ self.B.T  # sum gamma b <b, x>

    def apply(self, X):
        """H X for a row block X [n_vec, N]."""
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        return self.kinetic(X) + self.V[None, :] * X + self.nonlocal_(X)


def kinetic_1d(n, h):
    """Dense 1D kinetic matrix on a periodic line: T[i,j] = (1/n) sum_m G_m^2/2 cos(G_m (i-j) h)."""
    m = np.fft.fftfreq(n) * n
    G = 2.0 * np.pi * m / (n * h)
    idx = np.arange(n)
    D = (idx[:, None] - idx[None, :]) * h
    return (0.5 * (G[None, None, :] ** 2) * np.cos(G[None, None, :] * D[:, :, None])).sum(-1) / n


def dense_matrix(op: LocalOperator):
    """Explicit H (N x N) built as a Kronecker sum of 1D kinetic matrices plus diag(V) and the projectors."""
    nx, ny, nz = op.Qn
    Tx, Ty, Tz = kinetic_1d(nx, op.h[0]), kinetic_1d(ny, op.h[1]), kinetic_1d(nz, op.h[2])
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    H = (np.kron(np.kron(Tz, Iy), Ix) + np.kron(np.kron(Iz, Ty), Ix) + np.kron(np.kron(Iz, Iy), Tx))
    H += np.diag(op.V)
    if op.B.shape[1]:
        H += (op.B * op.gamma) @ op.B.T * op.dV
    return H
