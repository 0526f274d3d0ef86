"""Writes c2_dg.json: the assembled DG Hamiltonian of the 8x8-element slab (config 2) from the FP64 oracle.

Every one of the 64 elements is solved (Eq. LocalKS, Alg. CheFSI to residual 1e-10, Sec. II.A.1 ALBs by
SVD); the interior-penalty blocks (Eq. DGHamiltonian, alpha = 20, element plus 4 face neighbours) are
assembled into the dense N_b x N_b matrix (N_b = 64 x 32 = 2048, Eq. DGEigenvalue) and stored are:

* the lowest 64 eigenvalues of that matrix;
* for every element, the eigenvalues of its diagonal block and the singular values of its four
  off-diagonal blocks (basis-invariant: an orthogonal change of ALB basis inside an element leaves them
  unchanged);
* the largest asymmetry |H - H^T| of the assembled matrix;
* the DG solution of the lowest 64 states with 32 electrons at kT = 0.005 Ha (Eq. density with the diagonal
  density-matrix blocks, the band energy of Eq. DGvar, the Hellmann-Feynman gradient of Eq. hfforce at
  fixed ALBs): band energy, mu, the integral of the density, its values at 64 seeded grid points, and the
  atom gradient.

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
DG_NEL, DG_KT = 32.0, 0.005
PROBE_SEED = 5151


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
    return k, ik, info, dict(A=r["A"], dV=r["dV"])


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
    sols = {}
    for k, ik, info, sol in rows:
        ingr[k], infos[k], sols[k] = ik, info, sol
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
    from oracle import dg_solve
    from workloads.configs import probe_points
    eps, V = np.linalg.eigh(0.5 * (H + H.T))
    C = V[:, :N_LOW].T
    rho_e, mu, e_band = dg_solve.dg_density(p, sols, q.n_alb, eps[:N_LOW], C, DG_NEL, DG_KT)
    E2, mu2, gR = dg_solve.dg_band_gradient(p, sols, q.n_alb, eps[:N_LOW], C, DG_NEL, DG_KT)
    rho = np.zeros(p.v_extra.size)
    for k in range(M):
        dom = int(p.elem_dom[k])
        n = p.dom_n[dom]
        En = p.elem_En[k]
        gE = [np.mod(p.elem_E0[k][a] + np.arange(int(En[a])), n[a]) for a in range(3)]
        flat = (gE[2][:, None, None] * n[1] + gE[1][None, :, None]) * n[0] + gE[0][None, None, :]
        rho[int(p.dom_voff[dom]) + flat.ravel()] += rho_e[k]
    pts = probe_points(64, rho.size, PROBE_SEED)
    dV = float(np.prod(p.dom_h[0]))
    solution = {"n_states": N_LOW, "n_electrons": DG_NEL, "kT": DG_KT, "band_energy": float(e_band), "mu": float(mu),
                "band_energy_from_gradient_routine": float(E2), "rho_integral": float(rho.sum() * dV),
                "probe_seed": PROBE_SEED, "rho_points": [int(i) for i in pts],
                "rho_at_points": [float(v) for v in rho[pts]], "rho_max": float(rho.max()),
                "grad_R": [[float(v) for v in row] for row in gR]}
    doc = {"what": "oracle assembled DG Hamiltonian of the 8x8-element slab (config 2)",
           "cites": "Eq. LocalKS, Alg. CheFSI, Sec. II.A.1 (ALB by SVD), Eq. DGHamiltonian, Eq. DGEigenvalue",
           "oracle_settings": {"cheb_degree": DEGREE, "tol": TOL, "max_iter": MAX_ITER},
           "alpha": wl.alpha, "n_stencil": int(p.n_stencil), "N_b": int(H.shape[0]),
           "asymmetry_max": asym, "dropped_nonlocal_norm": dropped,
           "lowest_eigenvalues": [float(v) for v in lam[:N_LOW]],
           "eig_gap_abs_min": float(min(i["eig_gap_abs"] for i in infos)),
           "sv_relgap_min": float(min(i["sv_relgap"] for i in infos)),
           "max_resid": float(max(i["max_resid"] for i in infos)),
           "dg_solution": solution,
           "blocks": per}
    with open(os.path.join(HERE, "c2_dg.json"), "w") as f:
        json.dump(doc, f, indent=0)
    print("wrote c2_dg.json; lowest", lam[:4], "asym", asym)


if __name__ == "__main__":
    main()
