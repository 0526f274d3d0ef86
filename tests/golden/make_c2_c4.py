"""Writes c2_samples.json and c4_gradient.json from the FP64 oracle.

c2 (8x8 elements of 32x32x48, 40 eigenpairs, 32 ALBs): for sampled elements, the eigenvalues
(Eq. LocalKS, Alg. CheFSI, residual 1e-10), the singular values of the restricted block and the
eigenvalues of the diagonal DG block (Sec. II.A.1, Eq. DGHamiltonian), with the gaps that bound how
well the ALB subspace is defined.

c4 (the c2 geometry with its own seed and 48 eigenpairs, Fermi smearing kT = 0.01 Ha): every element is solved and
the band energy and its Hellmann-Feynman gradient (the local analogue of Eq. hfforce) are formed;
stored are the per-element energies, the atom gradient, and the V_eff gradient through its norm,
its sum, its projections on 4 seeded unit vectors and its values at 64 seeded grid points.

Only ``oracle/`` and the input generators are called.  Run from the repository root:
    python tests/golden/make_c2_c4.py
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

C2_SAMPLES = [0, 9, 27, 36, 50, 63]
DEGREE, TOL, MAX_ITER = 30, 1e-10, 150
PROBE_SEED = 4242


def solve(args):
    cfg, k, keep = args
    from workloads import make_config
    from oracle import driver, dg
    wl = make_config(cfg)
    wl.params.cheb_degree = DEGREE
    p, q = wl.problem, wl.params
    r = driver.solve_element(p, q, k, tol=TOL, max_iter=MAX_ITER)
    n_eig, n_alb = r["n_eig"], r["n_alb"]
    theta, s = r["theta"], r["sing"]
    out = dict(element=k, iters=int(r["iters"]), max_resid=float(r["resid"][:n_eig].max()),
               eigval=[float(v) for v in theta[:n_eig]], sing=[float(v) for v in s[:n_eig]],
               eig_gap_abs=float(theta[n_eig] - theta[n_eig - 1]), b_up=float(r["b_up"]),
               sv_relgap=float((s[n_alb - 1] - s[n_alb]) / s[0]))
    if cfg == 2:
        ik = dg.element_ingredients(p, k, r["X"][:n_eig], r["C"], r["A"])
        blk = dg.diagonal_block(p, k, ik, wl.alpha)
        out["dg_diag_eig"] = [float(v) for v in np.linalg.eigvalsh(0.5 * (blk + blk.T))]
    if keep:
        out["_sol"] = r
    return out


def main():
    from workloads import make_config
    from workloads.configs import electrons_per_element, probe_directions, probe_points
    from oracle import driver
    ctx = mp.get_context("spawn")
    M4 = make_config(4).problem.n_elem
    with ctx.Pool(os.cpu_count() or 1) as pool:
        rows2 = pool.map(solve, [(2, k, False) for k in C2_SAMPLES])
    doc2 = {"what": "oracle values for sampled elements of the 8x8-element slab (config 2)",
            "cites": "Eq. LocalKS, Alg. CheFSI, Sec. II.A.1 (ALB by SVD), Eq. DGHamiltonian (diagonal block)",
            "oracle_settings": {"cheb_degree": DEGREE, "tol": TOL, "max_iter": MAX_ITER},
            "samples": rows2}
    with open(os.path.join(HERE, "c2_samples.json"), "w") as f:
        json.dump(doc2, f, indent=1)
    with ctx.Pool(os.cpu_count() or 1) as pool:
        rows4 = pool.map(solve, [(4, k, True) for k in range(M4)])
    wl = make_config(4)
    p = wl.problem
    sols = {r["element"]: r["_sol"] for r in rows4}
    nel = electrons_per_element(p)
    E, gv, gR = driver.alb_grad(p, sols, wl.kT, nel)
    dirs = probe_directions(4, gv.size, PROBE_SEED)
    pts = probe_points(64, gv.size, PROBE_SEED + 1)
    doc4 = {"what": "oracle band energy and gradient of the config-4 slab (8x8 elements, kT 0.01 Ha)",
            "cites": "Eq. LocalKS, Alg. CheFSI; band energy with Fermi smearing and its Hellmann-Feynman "
                     "gradient (local analogue of Eq. hfforce)",
            "oracle_settings": {"cheb_degree": DEGREE, "tol": TOL, "max_iter": MAX_ITER},
            "kT": wl.kT, "probe_seed": PROBE_SEED,
            "energy": [float(v) for v in E], "n_electrons": [float(v) for v in nel],
            "grad_R": [[float(v) for v in row] for row in gR],
            "grad_v_norm": float(np.linalg.norm(gv)), "grad_v_sum": float(gv.sum()),
            "grad_v_proj": [float(v) for v in dirs @ gv],
            "grad_v_points": [int(i) for i in pts], "grad_v_at_points": [float(v) for v in gv[pts]],
            "eig_gap_abs_min": float(min(r["eig_gap_abs"] for r in rows4)),
            "max_resid": float(max(r["max_resid"] for r in rows4))}
    with open(os.path.join(HERE, "c4_gradient.json"), "w") as f:
        json.dump(doc4, f, indent=1)
    print("wrote c2_samples.json, c4_gradient.json")


if __name__ == "__main__":
    main()
