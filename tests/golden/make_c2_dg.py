"""Writes c2_dg.json: the assembled DG Hamiltonian of the 8x8-element slab (config 2) from the FP64 oracle.

Every one of the 64 elements is solved (Eq. LocalKS, Alg. CheFSI to residual 1e-10, Sec. II.A.1 ALBs by
SVD); the interior-penalty blocks (Eq. DGHamiltonian, alpha = 20, element plus 4 face neighbours) are
assembled into the dense N_b x N_b matrix (N_b = 64 x 32 = 2048, Eq. DGEigenvalue) and stored are:

* the lowest 64 eigenvalues of that matrix;
* for every element, the eigenvalues of its diagonal block and the singular values of its four
  off-diagonal blocks (basis-invariant: an orthogonal change of ALB basis inside an element leaves them
  unchanged);
* the largest asymmetry |H - H^T| of the assembled matrix.

Only ``oracle/`` and the input generators are called.  Run from the repository root:
    python tests/golden/make_c2_dg.py
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

DEGREE, TOL, MAX_ITER = 30, 1e-10, 150
N_LOW = 64


def solve(k):
    from workloads import make_config
    from oracle import driver, dg
    wl = make_config(2)
    wl.params.cheb_degree = DEGREE
    p, q = wl.problem, wl.params
    r = driver.solve_element(p, q, k, tol=TOL, max_iter=MAX_ITER)
    n_eig = r["n_eig"]
    ik = dg.element_ingredients(p, k, r["X"][:n_eig], r["C"], r["A"])
    info = dict(element=k, iters=int(r["iters"]), max_resid=float(r["resid"][:n_eig].max()),
                eig_gap_abs=float(r["theta"][n_eig] - r["theta"][n_eig - 1]),
                sv_relgap=float((r["sing"][r["n_alb"] - 1] - r["sing"][r["n_alb"]]) / r["sing"][0]))
    return k, ik, info


def main():
    from workloads import make_config
    from oracle import dg
    wl = make_config(2)
    p, q = wl.problem, wl.params
    M = p.n_elem
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        rows = pool.map(solve, range(M))
    ingr = [None] * M
    infos = [None] * M
    for k, ik, info in rows:
        ingr[k], infos[k] = ik, info
    blocks, dropped = dg.assemble(p, ingr, wl.alpha)
    H = dg.dense(p, blocks, q.n_alb)
    asym = float(np.abs(H - H.T).max())
    lam = np.linalg.eigvalsh(0.5 * (H + H.T))
    per = []
    for k in range(M):
        na = int(q.n_alb[k])
        B0 = blocks[k, 0, :na, :na]
        row = dict(element=k, diag_eig=[float(v) for v in np.linalg.eigvalsh(0.5 * (B0 + B0.T))], offdiag_sv=[])
        for s in range(1, p.n_stencil):
            kp = int(p.neighbors[k, s])
            Bs = blocks[k, s, :na, :int(q.n_alb[kp])]
            row["offdiag_sv"].append([float(v) for v in np.linalg.svd(Bs, compute_uv=False)])
        per.append(row)
    doc = {"what": "oracle assembled DG Hamiltonian of the 8x8-element slab (config 2)",
           "cites": "Eq. LocalKS, Alg. CheFSI, Sec. II.A.1 (ALB by SVD), Eq. DGHamiltonian, Eq. DGEigenvalue",
           "oracle_settings": {"cheb_degree": DEGREE, "tol": TOL, "max_iter": MAX_ITER},
           "alpha": wl.alpha, "n_stencil": int(p.n_stencil), "N_b": int(H.shape[0]),
           "asymmetry_max": asym, "dropped_nonlocal_norm": dropped,
           "lowest_eigenvalues": [float(v) for v in lam[:N_LOW]],
           "eig_gap_abs_min": float(min(i["eig_gap_abs"] for i in infos)),
           "sv_relgap_min": float(min(i["sv_relgap"] for i in infos)),
           "max_resid": float(max(i["max_resid"] for i in infos)),
           "blocks": per}
    with open(os.path.join(HERE, "c2_dg.json"), "w") as f:
        json.dump(doc, f, indent=0)
    print("wrote c2_dg.json; lowest", lam[:4], "asym", asym)


if __name__ == "__main__":
    main()
