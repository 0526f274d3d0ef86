"""Writes c3_samples.json: oracle values for sampled elements of the uneven batch (config 3).

Config 3 holds 256 independent elements whose extended grids are drawn from {24,32,40}^2 x {32,48},
with 2-6 atoms and 20-60 ALBs each.  For one element of each of six shapes the FP64 oracle solves
the local problem (Eq. LocalKS, Alg. CheFSI) to a residual of 1e-10, truncates to the ALBs
(Sec. II.A.1) and forms the diagonal DG block (Eq. DGHamiltonian).  Stored: eigenvalues, singular
values, diagonal-block eigenvalues and the gaps that bound how well the ALB subspace is defined.

Only ``oracle/`` and the input generators are called.  Run from the repository root:
    python tests/golden/make_c3_samples.py
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

import json
import multiprocessing as mp
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))

SHAPES = [(40, 40, 48), (24, 24, 32), (32, 24, 48), (40, 24, 32), (24, 40, 48), (32, 32, 32)]
DEGREE, TOL, MAX_ITER = 30, 1e-10, 150


def one(k):
    from workloads import make_config
    from oracle import driver, dg
    wl = make_config(3)
    wl.params.cheb_degree = DEGREE
    p, q = wl.problem, wl.params
    r = driver.solve_element(p, q, k, tol=TOL, max_iter=MAX_ITER)
    n_eig, n_alb = r["n_eig"], r["n_alb"]
    theta, s = r["theta"], r["sing"]
    ik = dg.element_ingredients(p, k, r["X"][:n_eig], r["C"], r["A"])
    blk = dg.diagonal_block(p, k, ik, wl.alpha)
    return dict(element=k, shape=[int(v) for v in p.elem_Qn[k]], n_eig=n_eig, n_alb=n_alb,
                iters=int(r["iters"]), max_resid=float(r["resid"][:n_eig].max()),
                eigval=[float(v) for v in theta[:n_eig]], sing=[float(v) for v in s[:n_eig]],
                dg_diag_eig=[float(v) for v in np.linalg.eigvalsh(0.5 * (blk + blk.T))],
                eig_gap_abs=float(theta[n_eig] - theta[n_eig - 1]), b_up=float(r["b_up"]),
                sv_relgap=float((s[n_alb - 1] - s[n_alb]) / s[0]))


def main():
    from workloads import make_config
    p = make_config(3).problem
    picks = []
    for sh in SHAPES:
        picks.append(int(next(k for k in range(p.n_elem) if tuple(int(v) for v in p.elem_Qn[k]) == sh)))
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(picks), os.cpu_count() or 1)) as pool:
        rows = pool.map(one, picks)
    doc = {"what": "oracle values for sampled elements of the uneven batch (config 3)",
           "cites": "Eq. LocalKS, Alg. CheFSI, Sec. II.A.1 (ALB by SVD), Eq. DGHamiltonian (diagonal block)",
           "oracle_settings": {"cheb_degree": DEGREE, "tol": TOL, "max_iter": MAX_ITER},
           "samples": rows}
    with open(os.path.join(HERE, "c3_samples.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote c3_samples.json")


if __name__ == "__main__":
    main()
