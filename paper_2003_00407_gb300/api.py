"""Python binding of libdgdft: argument marshalling only.

Every step of the computation runs in the CUDA library; this module turns a
``workloads.Problem`` / ``workloads.Params`` pair and torch device tensors
into the C structures of include/dgdft.h and back.  It raises when the
library is missing or a call fails; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi


class DgdftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_abi.STATUS_NAMES[code] if 0 <= code < len(_abi.STATUS_NAMES) else code}: {msg}")
        self.code = code


def _i32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _ptr(arr, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


class Marshalled:
    """Keeps the numpy buffers alive while the C structures point into them."""

    def __init__(self, prob, params, *, precision, cheb_degree, tol, max_iter, tol_mixed=0.0,
                 lanczos_steps=10, seed=None, flags=0, v_extra=None, x0=None, solver=0):
        self.keep = []

        def keep(a):
            self.keep.append(a)
            return a

        p = _abi.Problem()
        p.n_dom = int(prob.dom_n.shape[0])
        p.dom_n = _ptr(keep(_i32(prob.dom_n)), C.c_int)
        p.dom_h = _ptr(keep(_f64(prob.dom_h)), C.c_double)
        p.dom_voff = _ptr(keep(np.ascontiguousarray(prob.dom_voff, dtype=np.int64)), C.c_int64)
        p.v_extra = C.c_void_p(0 if v_extra is None else v_extra)
        p.n_elem = int(prob.n_elem)
        p.elem_dom = _ptr(keep(_i32(prob.elem_dom)), C.c_int)
        p.elem_E0 = _ptr(keep(_i32(prob.elem_E0)), C.c_int)
        p.elem_En = _ptr(keep(_i32(prob.elem_En)), C.c_int)
        p.elem_Qn = _ptr(keep(_i32(prob.elem_Qn)), C.c_int)
        p.neighbors = _ptr(keep(_i32(prob.neighbors)), C.c_int)
        p.n_stencil = int(prob.n_stencil)
        p.n_atoms = int(prob.n_atoms)
        p.atom_dom = _ptr(keep(_i32(prob.atom_dom if prob.n_atoms else np.zeros(1))), C.c_int)
        p.atom_pos = _ptr(keep(_f64(prob.atom_pos if prob.n_atoms else np.zeros(3))), C.c_double)
        p.well_depth = _ptr(keep(_f64(prob.well_depth if prob.n_atoms else np.zeros(1))), C.c_double)
        p.well_width = _ptr(keep(_f64(prob.well_width if prob.n_atoms else np.ones(1))), C.c_double)
        p.n_proj_per_atom = int(prob.n_proj_per_atom)
        pg = prob.proj_gamma if prob.proj_gamma.size else np.zeros(1)
        p.proj_gamma = _ptr(keep(_f64(pg)), C.c_double)
        p.proj_width = _ptr(keep(_f64(prob.proj_width if prob.n_atoms else np.ones(1))), C.c_double)
        p.r_cut = float(prob.r_cut)
        self.prob = p
        q = _abi.AlbParams()
        q.n_eig = _ptr(keep(_i32(params.n_eig)), C.c_int)
        q.n_alb = _ptr(keep(_i32(params.n_alb)), C.c_int)
        q.n_blk = _ptr(keep(_i32(params.n_blk)), C.c_int)
        q.cheb_degree = int(cheb_degree)
        q.tol = float(tol)
        q.tol_mixed = float(tol_mixed)
        q.max_iter = int(max_iter)
        q.lanczos_steps = int(lanczos_steps)
        q.precision = int(precision)
        q.seed = int(params.seed if seed is None else seed)
        q.flags = int(flags)
        q.x0 = C.c_void_p(0 if x0 is None else x0)
        q.solver = int(solver)
        self.params = q


class Context:
    """A libdgdft context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = _abi.load()
        h = C.c_void_p()
        r = self.lib.dgdft_ctx_create(C.byref(h), int(device))
        if r != 0:
            raise DgdftError(r, "dgdft_ctx_create: " + self.lib.dgdft_last_error(None).decode())
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.dgdft_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, r, allow=(0,)):
        if r not in allow:
            raise DgdftError(r, self.lib.dgdft_last_error(self.h).decode())
        return r


def query_sizes(m: Marshalled):
    out = (C.c_int64 * 6)()
    r = _abi.load().dgdft_alb_query_sizes(C.byref(m.prob), C.byref(m.params), out)
    if r != 0:
        raise DgdftError(r, "dgdft_alb_query_sizes: " + (_abi.load().dgdft_last_error(None) or b"").decode())
    return [int(v) for v in out]


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class ALBResult:
    eigval: torch.Tensor
    resid: torch.Tensor
    sing: torch.Tensor
    coef: torch.Tensor
    alb: torch.Tensor
    eigvec: torch.Tensor | None
    iters: torch.Tensor
    status: torch.Tensor
    L: int
    code: int
    struct: object = None
    history: np.ndarray = None

    def as_struct(self):
        s = _abi.AlbResult()
        for f in ("eigval", "resid", "sing", "coef", "alb", "iters", "status"):
            setattr(s, f, C.c_void_p(getattr(self, f).data_ptr()))
        s.eigvec = C.c_void_p(self.eigvec.data_ptr() if self.eigvec is not None else 0)
        s.history = C.c_void_p(self.history.ctypes.data if self.history is not None else 0)
        return s


def v_extra_tensor(prob, device="cuda"):
    return torch.as_tensor(np.ascontiguousarray(prob.v_extra, dtype=np.float64), device=device)


def alb_generate(ctx: Context, prob, params, *, precision=_abi.FP64, cheb_degree=None, tol=None, max_iter=None,
                 tol_mixed=0.0, keep_eigvec=True, v_extra=None, allow_not_converged=True, host_buffers=False,
                 x0=None, solver=_abi.CHEFSI):
    """ALB generation for every element (dgdft_alb_generate).  Returns ALBResult of device tensors.

    x0: optional warm start, a float64 tensor in the packed [n_eig][N] layout of ALBResult.eigvec (on the
    device, or in host memory with host_buffers)."""
    dev = torch.device("cuda", ctx.device)
    if v_extra is None:
        # device tensor, or (host buffers) a pinned host copy that the library stages itself
        v_extra = v_extra_tensor(prob, "cpu").pin_memory() if host_buffers else v_extra_tensor(prob, dev)
    m = Marshalled(prob, params, precision=precision,
                   cheb_degree=params.cheb_degree if cheb_degree is None else cheb_degree,
                   tol=params.tol if tol is None else tol,
                   max_iter=params.max_iter if max_iter is None else max_iter, tol_mixed=tol_mixed,
                   flags=_abi.HOST_BUFFERS if host_buffers else 0,
                   v_extra=None if v_extra is None else v_extra.data_ptr(),
                   x0=None if x0 is None else x0.data_ptr(), solver=solver)
    m.keep.append(v_extra)
    if x0 is not None:
        if x0.dtype != torch.float64 or not x0.is_contiguous():
            raise ValueError("x0 must be a contiguous float64 tensor in the eigvec layout")
        m.keep.append(x0)
    L, n_alb_tot, n_vec_tot, ncoef, _, _ = query_sizes(m)
    M = prob.n_elem
    kw = dict(dtype=torch.float64, device="cpu" if host_buffers else dev)
    if host_buffers:
        kw["pin_memory"] = True
    res = ALBResult(eigval=torch.empty(M, L, **kw), resid=torch.empty(M, L, **kw), sing=torch.empty(M, L, **kw),
                    coef=torch.empty(M, L, L, **kw), alb=torch.empty(max(1, n_alb_tot), **kw),
                    eigvec=(torch.empty(n_vec_tot, dtype=torch.float64, device=dev)
                            if keep_eigvec and not host_buffers else None),
                    iters=torch.empty(M, dtype=torch.int32, device=kw["device"], pin_memory=host_buffers),
                    status=torch.empty(M, dtype=torch.int32, device=kw["device"], pin_memory=host_buffers),
                    L=L, code=0)
    res.history = np.full(int(m.params.max_iter) + 2, -1.0)
    s = res.as_struct()
    allow = (0, _abi.NOT_CONVERGED) if allow_not_converged else (0,)
    res.code = ctx.check(ctx.lib.dgdft_alb_generate(ctx.h, C.byref(m.prob), C.byref(m.params), C.byref(s),
                                                    _stream()), allow)
    res.struct = (m, s)
    return res


def apply_hamiltonian(ctx: Context, prob, params, X: torch.Tensor, precision=_abi.FP64):
    """Y = H X for packed blocks of n_blk vectors per element (device tensors, float64 or float32)."""
    m = Marshalled(prob, params, precision=precision, cheb_degree=max(2, params.cheb_degree), tol=params.tol,
                   max_iter=params.max_iter, v_extra=v_extra_tensor(prob, X.device).data_ptr())
    m.keep.append(v := v_extra_tensor(prob, X.device))
    m.prob.v_extra = C.c_void_p(v.data_ptr())
    Y = torch.empty_like(X)
    ctx.check(ctx.lib.dgdft_apply_hamiltonian(ctx.h, C.byref(m.prob), C.byref(m.params), C.c_void_p(X.data_ptr()),
                                              C.c_void_p(Y.data_ptr()), _stream()))
    return Y


def gram_fp32(ctx: Context, X: torch.Tensor, x_off, nx, np_, dV, Y: torch.Tensor = None, y_off=None, ny=None,
              ldg=None):
    """G_k = dV_k X_k Y_k^T for packed FP32 blocks on the tensor cores (3xTF32); returns [n][ldg][ldg] FP64."""
    n = len(nx)
    if Y is None:
        Y, y_off, ny = X, x_off, nx
    nx_, ny_, npp = _i32(nx), _i32(ny), _i32(np_)
    dv = _f64(dV)
    xo = np.ascontiguousarray(x_off, dtype=np.int64)
    yo = np.ascontiguousarray(y_off, dtype=np.int64)
    ldg = int(ldg or max(1, int(max(nx_.max(initial=0), ny_.max(initial=0)))))
    G = torch.empty((n, ldg, ldg), dtype=torch.float64, device=X.device)
    ctx.check(ctx.lib.dgdft_gram_fp32(ctx.h, n, _ptr(nx_, C.c_int), _ptr(ny_, C.c_int), _ptr(npp, C.c_int),
                                      _ptr(dv, C.c_double), C.c_void_p(X.data_ptr()), _ptr(xo, C.c_int64),
                                      C.c_void_p(Y.data_ptr()), _ptr(yo, C.c_int64), C.c_void_p(G.data_ptr()), ldg,
                                      _stream()))
    return G


def rotate_fp32(ctx: Context, X: torch.Tensor, x_off, nin, np_, W: torch.Tensor, nout, Z: torch.Tensor = None,
                z_off=None):
    """Z_k = W_k^T X_k for packed FP32 blocks on the tensor cores (3xTF32); W [n][ldw][ldw] FP64 on the device.
    Z defaults to a new packed tensor with the output blocks back to back."""
    n = len(nin)
    ni, no, npp = _i32(nin), _i32(nout), _i32(np_)
    xo = np.ascontiguousarray(x_off, dtype=np.int64)
    if Z is None:
        sizes = no.astype(np.int64) * npp
        z_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        Z = torch.empty(int(sizes.sum()), dtype=torch.float32, device=X.device)
    zo = np.ascontiguousarray(z_off, dtype=np.int64)
    ctx.check(ctx.lib.dgdft_rotate_fp32(ctx.h, n, _ptr(ni, C.c_int), _ptr(no, C.c_int), _ptr(npp, C.c_int),
                                        C.c_void_p(X.data_ptr()), _ptr(xo, C.c_int64), C.c_void_p(W.data_ptr()),
                                        int(W.shape[-1]), C.c_void_p(Z.data_ptr()), _ptr(zo, C.c_int64), _stream()))
    return Z, zo


def chebyshev_filter(ctx: Context, prob, params, X: torch.Tensor, bounds: np.ndarray, degree: int,
                     precision=_abi.FP64):
    """Y = p_m(H) X with per-element bounds (a0, b_low, b_up)."""
    v = v_extra_tensor(prob, X.device)
    m = Marshalled(prob, params, precision=precision, cheb_degree=degree, tol=params.tol,
                   max_iter=params.max_iter, v_extra=v.data_ptr())
    m.keep.append(v)
    b = _f64(bounds)
    Y = torch.empty_like(X)
    ctx.check(ctx.lib.dgdft_chebyshev_filter(ctx.h, C.byref(m.prob), C.byref(m.params), _ptr(b, C.c_double),
                                             C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()), _stream()))
    return Y


def unpack_blocks(flat: torch.Tensor, counts, sizes):
    """Split a packed buffer into per-element [count, size] views."""
    out, o = [], 0
    for c, s in zip(counts, sizes):
        out.append(flat[o:o + c * s].view(c, s))
        o += c * s
    return out


def dg_assemble(ctx: Context, prob, params, res: ALBResult, alpha: float):
    """DG blocks [M, n_stencil, L, L] (dgdft_dg_assemble) from a result of alb_generate."""
    m, s = res.struct
    v = v_extra_tensor(prob, torch.device("cuda", ctx.device))
    m.keep.append(v)
    m.prob.v_extra = C.c_void_p(v.data_ptr())
    M, L = prob.n_elem, res.L
    blocks = torch.empty(M, int(prob.n_stencil), L, L, dtype=torch.float64, device=v.device)
    ctx.check(ctx.lib.dgdft_dg_assemble(ctx.h, C.byref(m.prob), C.byref(m.params), C.byref(s), float(alpha),
                                        C.c_void_p(blocks.data_ptr()), _stream()))
    return blocks


def alb_grad(ctx: Context, prob, params, res: ALBResult, kT: float, n_electrons):
    """(energy [M], grad_v [points of all domains], grad_R [n_atoms, 3]) (dgdft_alb_grad)."""
    m, s = res.struct
    dev = torch.device("cuda", ctx.device)
    nel = _f64(n_electrons)
    energy = torch.empty(prob.n_elem, dtype=torch.float64, device=dev)
    grad_v = torch.empty(int(prob.v_extra.size), dtype=torch.float64, device=dev)
    grad_R = torch.empty(max(1, prob.n_atoms), 3, dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.dgdft_alb_grad(ctx.h, C.byref(m.prob), C.byref(m.params), C.byref(s), float(kT),
                                     _ptr(nel, C.c_double), C.c_void_p(energy.data_ptr()),
                                     C.c_void_p(grad_v.data_ptr()), C.c_void_p(grad_R.data_ptr()), _stream()))
    return energy, grad_v, grad_R[:prob.n_atoms]


def alb_views(prob, params, res: ALBResult):
    """Per-element views: ALBs [n_alb, NE] and eigenvectors [n_eig, N] (if kept)."""
    NE = np.prod(prob.elem_En, axis=1)
    N = np.prod(prob.elem_Qn, axis=1)
    A = unpack_blocks(res.alb, params.n_alb, NE)
    X = unpack_blocks(res.eigvec, params.n_eig, N) if res.eigvec is not None else None
    return A, X


def dg_assemble_host(ctx: Context, prob, params, res: ALBResult, alpha: float):
    """dg_assemble with host buffers (coef and blocks in pinned host memory, eigenvectors kept in the context)."""
    m, s = res.struct
    m.params.flags = _abi.HOST_BUFFERS
    m.prob.v_extra = C.c_void_p(prob.v_extra.ctypes.data) if prob.v_extra is not None else C.c_void_p(0)
    M, L = prob.n_elem, res.L
    blocks = torch.empty(M, int(prob.n_stencil), L, L, dtype=torch.float64, pin_memory=True)
    ctx.check(ctx.lib.dgdft_dg_assemble(ctx.h, C.byref(m.prob), C.byref(m.params), C.byref(s), float(alpha),
                                        C.c_void_p(blocks.data_ptr()), _stream()))
    return blocks


class ALBBandEnergy(torch.autograd.Function):
    """Total Fermi-smeared band energy sum_k E_k of the local problems as a function of the global
    V_eff correction (v_extra) and the atom positions; the backward pass returns the gradient that
    dgdft_alb_grad forms (the local analogue of Eq. hfforce) in the same call as the forward energies.

    Usage: E = ALBBandEnergy.apply(v_extra, atom_pos, ctx, prob, params, kT, n_electrons, options)
    with v_extra [total grid points] and atom_pos [n_atoms, 3] float64 tensors and options a dict of
    alb_generate keywords (precision, cheb_degree, tol, max_iter)."""

    @staticmethod
    def forward(fctx, v_extra, atom_pos, ctx, prob, params, kT, n_electrons, options):
        import copy
        dev = torch.device("cuda", ctx.device)
        p = copy.copy(prob)
        p.atom_pos = atom_pos.detach().to("cpu", torch.float64).numpy().copy()
        p.v_extra = v_extra.detach().to("cpu", torch.float64).numpy().reshape(-1).copy()
        v_dev = v_extra.detach().to(dev, torch.float64).reshape(-1).contiguous()
        res = alb_generate(ctx, p, params, v_extra=v_dev, keep_eigvec=True, **(options or {}))
        energy, grad_v, grad_R = alb_grad(ctx, p, params, res, kT, n_electrons)
        fctx.save_for_backward(grad_v, grad_R)
        fctx.shapes = (v_extra.shape, v_extra.device, atom_pos.device)
        return energy.sum()

    @staticmethod
    def backward(fctx, g):
        grad_v, grad_R = fctx.saved_tensors
        vshape, vdev, rdev = fctx.shapes
        return ((g * grad_v).reshape(vshape).to(vdev), (g * grad_R).to(rdev), None, None, None, None, None, None)


def dg_layout(prob, params):
    """(tr_off [M+1], pe_off [M+1]) int64: offsets of the per-element DG ingredient records
    (dgdft_dg_query_layout, host only)."""
    m = Marshalled(prob, params, precision=_abi.FP64, cheb_degree=max(2, params.cheb_degree), tol=params.tol,
                   max_iter=params.max_iter)
    M = prob.n_elem
    tr = np.zeros(M + 1, dtype=np.int64)
    pe = np.zeros(M + 1, dtype=np.int64)
    lib = _abi.load()
    r = lib.dgdft_dg_query_layout(C.byref(m.prob), C.byref(m.params), _ptr(tr, C.c_int64), _ptr(pe, C.c_int64))
    if r != 0:
        raise DgdftError(r, "dgdft_dg_query_layout: " + (lib.dgdft_last_error(None) or b"").decode())
    return tr, pe


def dg_ingredients(ctx: Context, prob, params, res: ALBResult):
    """(kv [M, L, L], traces [tr_off[M]], proj [pe_off[M]]) device tensors (dgdft_dg_ingredients)."""
    m, s = res.struct
    dev = torch.device("cuda", ctx.device)
    v = v_extra_tensor(prob, dev)
    m.keep.append(v)
    m.prob.v_extra = C.c_void_p(v.data_ptr())
    tr, pe = dg_layout(prob, params)
    M, L = prob.n_elem, res.L
    kv = torch.empty(M, L, L, dtype=torch.float64, device=dev)
    traces = torch.zeros(max(1, int(tr[-1])), dtype=torch.float64, device=dev)
    proj = torch.zeros(max(1, int(pe[-1])), dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.dgdft_dg_ingredients(ctx.h, C.byref(m.prob), C.byref(m.params), C.byref(s),
                                           C.c_void_p(kv.data_ptr()), C.c_void_p(traces.data_ptr()),
                                           C.c_void_p(proj.data_ptr()), _stream()))
    return kv, traces, proj


def dg_blocks(ctx: Context, prob, params, kv, traces, proj, alpha: float):
    """DG blocks [M, n_stencil, L, L] from ingredient arrays (dgdft_dg_blocks); L = kv.shape[1]."""
    dev = torch.device("cuda", ctx.device)
    m = Marshalled(prob, params, precision=_abi.FP64, cheb_degree=max(2, params.cheb_degree), tol=params.tol,
                   max_iter=params.max_iter)
    M, L = prob.n_elem, int(kv.shape[1])
    blocks = torch.empty(M, int(prob.n_stencil), L, L, dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.dgdft_dg_blocks(ctx.h, C.byref(m.prob), C.byref(m.params), C.c_void_p(kv.data_ptr()),
                                      C.c_void_p(traces.data_ptr()), C.c_void_p(proj.data_ptr()), float(alpha),
                                      C.c_void_p(blocks.data_ptr()), _stream()))
    return blocks


def result_subset(res: ALBResult, prob, params, elems, sub_prob, sub_params, precision=_abi.FP64):
    """The part of an alb_generate result that belongs to `elems` (in that order), as a result of the
    sub-problem (sub_prob, sub_params) over those elements: per-element rows and packed records are
    copied (device tensors); the eigenvectors must have been kept."""
    if res.eigvec is None:
        raise ValueError("result_subset needs the eigenvectors (alb_generate(keep_eigvec=True))")
    elems = np.asarray(elems, dtype=np.int64)
    NE = np.prod(prob.elem_En, axis=1).astype(np.int64)
    N = np.prod(prob.elem_Qn, axis=1).astype(np.int64)
    a_off = np.concatenate([[0], np.cumsum(params.n_alb.astype(np.int64) * NE)])
    e_off = np.concatenate([[0], np.cumsum(params.n_eig.astype(np.int64) * N)])
    idx = torch.as_tensor(elems, device=res.eigval.device)
    m = Marshalled(sub_prob, sub_params, precision=precision, cheb_degree=max(2, sub_params.cheb_degree),
                   tol=sub_params.tol, max_iter=sub_params.max_iter)
    L = query_sizes(m)[0]
    if L != res.L:
        raise ValueError("the sub-problem's row length differs from the result's")
    cat = lambda t, off: torch.cat([t[int(off[k]):int(off[k + 1])] for k in elems]) if len(elems) else t[:0]
    sub = ALBResult(eigval=res.eigval[idx].contiguous(), resid=res.resid[idx].contiguous(),
                    sing=res.sing[idx].contiguous(), coef=res.coef[idx].contiguous(),
                    alb=cat(res.alb, a_off).contiguous(), eigvec=cat(res.eigvec, e_off).contiguous(),
                    iters=res.iters[idx].contiguous(), status=res.status[idx].contiguous(), L=L, code=res.code)
    sub.struct = (m, sub.as_struct())
    return sub


def dg_eigensolve(ctx: Context, prob, params, blocks: torch.Tensor, n_states: int, n_blk: int, *,
                  cheb_degree=30, tol=1e-10, max_iter=200, lanczos_steps=10, seed=None, keep_vectors=True,
                  allow_not_converged=False):
    """Lowest eigenpairs of the assembled DG Hamiltonian from its stencil blocks (dgdft_dg_eigensolve).

    Returns (eigval [n_blk], resid [n_blk], eigvec [n_blk, N_b] or None, passes) on the device."""
    dev = torch.device("cuda", ctx.device)
    m = Marshalled(prob, params, precision=_abi.FP64, cheb_degree=max(2, params.cheb_degree), tol=params.tol,
                   max_iter=params.max_iter)
    sp = _abi.DGSolveParams(n_states=int(n_states), n_blk=int(n_blk), cheb_degree=int(cheb_degree), tol=float(tol),
                            max_iter=int(max_iter), lanczos_steps=int(lanczos_steps),
                            seed=int(params.seed if seed is None else seed))
    Nb = int(np.sum(params.n_alb))
    ev = torch.empty(n_blk, dtype=torch.float64, device=dev)
    rs = torch.empty(n_blk, dtype=torch.float64, device=dev)
    vec = torch.empty(n_blk, Nb, dtype=torch.float64, device=dev) if keep_vectors else None
    it = torch.zeros(1, dtype=torch.int32, device=dev)
    blocks = blocks.contiguous()
    allow = (0, _abi.NOT_CONVERGED) if allow_not_converged else (0,)
    ctx.check(ctx.lib.dgdft_dg_eigensolve(ctx.h, C.byref(m.prob), C.byref(m.params), C.c_void_p(blocks.data_ptr()),
                                          C.byref(sp), C.c_void_p(ev.data_ptr()), C.c_void_p(rs.data_ptr()),
                                          C.c_void_p(vec.data_ptr() if vec is not None else 0),
                                          C.c_void_p(it.data_ptr()), _stream()), allow)
    return ev, rs, vec, int(it.item())


def dg_density(ctx: Context, prob, params, res: ALBResult, eigval: torch.Tensor, eigvec: torch.Tensor, n: int,
               n_electrons: float, kT: float, forces=True):
    """(rho [total grid points], band energy, mu, grad_R [n_atoms, 3] or None) of the DG solution
    (dgdft_dg_density): density from the diagonal density-matrix blocks, band energy, dE/dR at fixed ALBs."""
    m, s = res.struct
    dev = torch.device("cuda", ctx.device)
    rho = torch.empty(int(prob.v_extra.size), dtype=torch.float64, device=dev)
    em = torch.empty(2, dtype=torch.float64, device=dev)
    gR = torch.empty(max(1, prob.n_atoms), 3, dtype=torch.float64, device=dev) if forces else None
    ev = eigval.contiguous()
    vec = eigvec.contiguous()
    ctx.check(ctx.lib.dgdft_dg_density(ctx.h, C.byref(m.prob), C.byref(m.params), C.byref(s),
                                       C.c_void_p(ev.data_ptr()), C.c_void_p(vec.data_ptr()), int(n),
                                       float(n_electrons), float(kT), C.c_void_p(rho.data_ptr()),
                                       C.c_void_p(em.data_ptr()), C.c_void_p(gR.data_ptr() if forces else 0),
                                       _stream()))
    e = em.cpu().numpy()
    return rho, float(e[0]), float(e[1]), (gR[:prob.n_atoms] if forces else None)
