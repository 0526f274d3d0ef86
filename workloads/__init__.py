"""Seeded synthetic DGDFT workloads (inputs only).

This package builds the problem descriptions that both the CPU oracle and the
CUDA library consume: periodic domains, the element partition (Sec. II.A,
"Discontinuous Galerkin density functional theory"), atom positions with
Gaussian local wells and Kleinman-Bylander projector coefficients (Eq.
LocalKS), ALB counts and solver parameters.  It holds none of the method's
arithmetic: no potential, projector, Hamiltonian or eigen-solver evaluation
lives here, only random draws and geometry bookkeeping.
"""
from .problem import Problem, Params, Workload, STENCIL_SELF, STENCIL_X, STENCIL_XY, STENCIL_XYZ, STENCIL_XY9
from .configs import make_config, CONFIG_NAMES, n_blk_rule

__all__ = ["Problem", "Params", "Workload", "make_config", "CONFIG_NAMES", "n_blk_rule",
           "STENCIL_SELF", "STENCIL_X", "STENCIL_XY", "STENCIL_XYZ", "STENCIL_XY9"]
