"""The oracle over every element of a workload (ALB generation, DG assembly, gradient)."""
from __future__ import annotations

import numpy as np

from . import local_operator as lo
from . import chefsi as cf
from . import alb as al
from . import dg as dgm
from . import grad as gr


def solve_element(prob, params, k, tol=None, max_iter=None, dense_route=False):
    """Eigenpairs, ALBs and coefficients of element k."""
    op = lo.LocalOperator(prob, k)
    n_eig, n_alb, n_blk = int(params.n_eig[k]), int(params.n_alb[k]), int(params.n_blk[k])
    tol = params.tol if tol is None else tol
    max_iter = params.max_iter if max_iter is None else max_iter
    if dense_route:
        H = lo.dense_matrix(op)
        lam, V = np.linalg.eigh(H)
        X = V[:, :n_blk].T / np.sqrt(op.dV)
        theta = lam[:n_blk]
        HX = op.apply(X)
        resid = np.sqrt(((HX - theta[:, None] * X) ** 2).sum(1) * op.dV)
        res = dict(theta=theta, X=X, resid=resid, iters=0, converged=True, b_up=float(lam[-1]))
    else:
        X0 = cf.random_block(params.seed, k, n_blk, op.N)
        res = cf.chefsi(op, n_eig, n_blk, params.cheb_degree, tol, max_iter, X0,
                        params.lanczos_steps)
    Qn, En = prob.elem_Qn[k], prob.elem_En[k]
    Phi_E = al.restrict(res["X"][:n_eig], Qn, lo.e_offset_in_q(prob, k), En)
    A, C, sing = al.svd_truncate(Phi_E, n_alb, op.dV)
    res.update(A=A, C=C, sing=sing, n_eig=n_eig, n_alb=n_alb, dV=op.dV)
    return res


def _solve_star(args):
    prob, params, k, tol, max_iter = args
    return solve_element(prob, params, k, tol=tol, max_iter=max_iter)


def alb_generate(prob, params, elems=None, tol=None, max_iter=None, processes=1):
    """Solve the listed elements (all by default); processes>1 uses a spawn pool."""
    elems = list(range(prob.n_elem)) if elems is None else list(elems)
    if processes > 1 and len(elems) > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes) as pool:
            out = pool.map(_solve_star, [(prob, params, k, tol, max_iter) for k in elems])
    else:
        out = [solve_element(prob, params, k, tol=tol, max_iter=max_iter) for k in elems]
    return dict(zip(elems, out))


def dg_assemble(prob, sols, alpha):
    """DG blocks for all elements from solve_element results (dict k -> result)."""
    ingr = [dgm.element_ingredients(prob, k, sols[k]["X"][:sols[k]["n_eig"]], sols[k]["C"], sols[k]["A"])
            for k in range(prob.n_elem)]
    return dgm.assemble(prob, ingr, alpha)


def alb_grad(prob, sols, kT, n_electrons):
    """(energy [M], grad_v [len(v_extra)], grad_R [n_atoms, 3]) from solve_element results."""
    grad_v = np.zeros_like(prob.v_extra)
    grad_R = np.zeros((prob.n_atoms, 3))
    E = np.zeros(prob.n_elem)
    for k in sorted(sols):
        s = sols[k]
        E[k] = gr.element_gradient(prob, k, s["theta"][:s["n_eig"]], s["X"][:s["n_eig"]],
                                   float(n_electrons[k]), kT, grad_v, grad_R)
    return E, grad_v, grad_R
