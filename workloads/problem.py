"""Problem and parameter records shared by the oracle and the CUDA library.

Geometry conventions (Sec. II.A, element partition and extended elements):

* A *domain* is a periodic box of ``n = (nx, ny, nz)`` grid points with spacing
  ``h``; grid point ``(i, j, k)`` sits at ``(i*hx, j*hy, k*hz)``.  Arrays over a
  domain are stored ``[z][y][x]`` (x fastest).
* Element ``E_k`` is the block of grid points ``E0 .. E0+En-1`` of its domain
  (indices wrap periodically).  The extended element ``Q_k`` has extent ``Qn``
  and is centred on ``E_k``: it starts at ``E0 - (Qn-En)//2`` (wrapping), so
  ``Qn - En`` must be even and ``Qn <= n``.
* ``neighbors[k, s]`` lists the element across stencil slot ``s``:
  slot 0 is ``k`` itself, then the faces ``-x, +x, -y, +y, -z, +z`` for as many
  axes as the stencil has faces, then (9-slot stencil only) the xy corners
  ``-x-y, +x-y, -x+y, +x+y`` which carry only nonlocal couplings.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# Stencil sizes: number of slots in ``neighbors`` and which faces exist.
STENCIL_SELF = 1   # independent elements, no faces
STENCIL_X = 3      # faces normal to x
STENCIL_XY = 5     # faces normal to x and y (2D partition; elements span z)
STENCIL_XYZ = 7    # faces normal to x, y and z (3D partition)
STENCIL_XY9 = 9    # x and y faces plus the four xy-corner neighbours

FACE_AXES = {STENCIL_SELF: 0, STENCIL_X: 1, STENCIL_XY: 2, STENCIL_XYZ: 3, STENCIL_XY9: 2}


@dataclass
class Problem:
    """Statement of the local Kohn-Sham problems and the DG partition."""
    dom_n: np.ndarray        # [n_dom, 3] int32, grid points per axis (x, y, z)
    dom_h: np.ndarray        # [n_dom, 3] float64, spacing (bohr)
    dom_voff: np.ndarray     # [n_dom] int64, offset of the domain's points in v_extra
    v_extra: np.ndarray      # [sum_d prod(dom_n[d])] float64, V_eff minus the wells (Ha)
    elem_dom: np.ndarray     # [M] int32
    elem_E0: np.ndarray      # [M, 3] int32
    elem_En: np.ndarray      # [M, 3] int32
    elem_Qn: np.ndarray      # [M, 3] int32
    neighbors: np.ndarray    # [M, n_stencil] int32, -1 = no element
    n_stencil: int
    atom_dom: np.ndarray     # [n_atoms] int32
    atom_pos: np.ndarray     # [n_atoms, 3] float64 (bohr, inside the domain box)
    well_depth: np.ndarray   # [n_atoms] float64 D_I (Ha)
    well_width: np.ndarray   # [n_atoms] float64 w_I (bohr), Gaussian sigma
    n_proj_per_atom: int     # 0 (no nonlocal term), 1 (s) or 4 (s, px, py, pz)
    proj_gamma: np.ndarray   # [n_atoms, n_proj_per_atom] float64 (Ha)
    proj_width: np.ndarray   # [n_atoms] float64 sigma of the projector radial Gaussian
    r_cut: float             # support radius of wells and projectors (bohr)

    @property
    def n_elem(self) -> int:
        return int(self.elem_dom.shape[0])

    @property
    def n_atoms(self) -> int:
        return int(self.atom_pos.shape[0])

    def domain_points(self, d: int) -> int:
        return int(np.prod(self.dom_n[d]))

    def v_extra_domain(self, d: int) -> np.ndarray:
        """v_extra of domain d as a [nz, ny, nx] view."""
        nx, ny, nz = (int(v) for v in self.dom_n[d])
        o = int(self.dom_voff[d])
        return self.v_extra[o:o + nx * ny * nz].reshape(nz, ny, nx)

    def q_points(self, k: int) -> int:
        return int(np.prod(self.elem_Qn[k]))

    def e_points(self, k: int) -> int:
        return int(np.prod(self.elem_En[k]))


@dataclass
class Params:
    """Solver parameters of the ALB generation (Alg. CheFSI, Sec. II.A)."""
    n_eig: np.ndarray        # [M] int32, eigenpairs kept (J_k before truncation)
    n_alb: np.ndarray        # [M] int32, ALBs kept after the SVD truncation
    n_blk: np.ndarray        # [M] int32, filter block = n_eig + guard vectors
    cheb_degree: int = 10    # m, the filter order (10..40 in Alg. CheFSI)
    tol: float = 1e-8        # residual tolerance, dV-norm of H x - lambda x
    max_iter: int = 60       # cap on subspace iterations
    seed: int = 20030407     # counter-based random start
    lanczos_steps: int = 10  # steps of the Lanczos upper-bound estimate


@dataclass
class Workload:
    name: str
    problem: Problem
    params: Params
    alpha: float = 20.0                  # interior-penalty parameter (Eq. DGHamiltonian)
    kT: float = 0.01                     # Fermi smearing temperature (Ha)
    n_electrons: np.ndarray = field(default_factory=lambda: np.zeros(0))  # [M]
    description: str = ""
