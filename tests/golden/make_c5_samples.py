"""Writes c5_samples.json: oracle values for sampled elements of the 32x32-element sheet.

For each sampled element of the 1024-element sheet (32x32x48 extended elements, 72
eigenpairs, 64 ALBs) the FP64 oracle solves the local problem (Eq. LocalKS, Alg. CheFSI)
to a residual of 1e-10, truncates to the ALBs (Sec. II.A.1) and forms the diagonal DG
block (Eq. DGHamiltonian, alpha as in the workload).  Stored: the eigenvalues, the
singular values of the restricted block, the eigenvalues of the diagonal DG block (basis
invariant), the gap after eigenvalue n_eig and the relative gaps that bound how well the ALB
subspace is defined.

Only ``oracle/`` and the input generators are called.  Run from the repository root:
    python tests/golden/make_c5_samples.py
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

SAMPLES = [0, 31, 100, 345, 512, 700, 993, 1023]
DEGREE, TOL, MAX_ITER = 40, 1e-10, 100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c5_samples.json")


def one(k):
    from workloads import make_config
    from oracle import driver, dg
    wl = make_config(5)
    wl.params.cheb_degree = DEGREE
    p, q = wl.problem, wl.params
    r = driver.solve_element(p, q, k, tol=TOL, max_iter=MAX_ITER)
    n_eig, n_alb, n_blk = r["n_eig"], r["n_alb"], int(q.n_blk[k])
    ik = dg.element_ingredients(p, k, r["X"][:n_eig], r["C"], r["A"])
    blk = dg.diagonal_block(p, k, ik, wl.alpha)
    theta = r["theta"]
    eig_gap_abs = float(theta[n_eig] - theta[n_eig - 1])
    eig_gap = eig_gap_abs / max(abs(float(r["b_up"])), 1e-300)
    s = r["sing"]
    sv_gap = float((s[n_alb - 1] - s[n_alb]) / s[0])
    return dict(element=k, iters=int(r["iters"]), max_resid=float(r["resid"][:n_eig].max()),
                eigval=[float(v) for v in theta[:n_eig]], sing=[float(v) for v in s[:n_eig]],
                dg_diag_eig=[float(v) for v in np.linalg.eigvalsh(0.5 * (blk + blk.T))],
                eig_gap_abs=eig_gap_abs, eig_relgap=eig_gap, b_up=float(r["b_up"]), sv_relgap=sv_gap, n_blk=n_blk)


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(SAMPLES), os.cpu_count() or 1)) as pool:
        rows = pool.map(one, SAMPLES)
    doc = {"what": "oracle values for sampled elements of the 1024-element sheet (config 5)",
           "cites": "Eq. LocalKS, Alg. CheFSI, Sec. II.A.1 (ALB by SVD), Eq. DGHamiltonian (diagonal block)",
           "oracle_settings": {"cheb_degree": DEGREE, "tol": TOL, "max_iter": MAX_ITER},
           "samples": rows}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
