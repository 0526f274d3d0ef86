"""Interior-penalty DG Hamiltonian blocks from the ALBs (Eq. DGHamiltonian).

H^DG_{k',j'; k,j} = ( 1/2 <grad phi_{k,j'}, grad phi_{k,j}>_T + <phi_{k,j'}, V_eff phi_{k,j}>_T ) delta_{kk'}
                  + sum_{I,l} gamma_{I,l} <phi_{k',j'}, b_{I,l}>_T <b_{I,l}, phi_{k,j}>_T
                  - 1/2 <[[phi_{k',j'}]], {{grad phi_{k,j}}}>_S - 1/2 <{{grad phi_{k',j'}}}, [[phi_{k,j}]]>_S
                  + alpha <[[phi_{k',j'}]], [[phi_{k,j}]]>_S

The paper defines neither the jump, the average, the face positions, the
quadrature nor the units of alpha.  Readings (standard symmetric interior
penalty DG on a cell-centred partition):

* element E occupies grid points [s, s+n_E) along each axis; its faces lie
  half a spacing outside the end points, so the elements tile the domain;
* an ALB is the restriction to E of psi = Phi^Q C, a trigonometric
  interpolant on Q; gradients on E are spectral derivatives on Q (Nyquist
  coefficient dropped) restricted to E; face values and normal derivatives
  evaluate the same interpolant on the half-shifted plane through 1D weights
  along the normal (Nyquist dropped, which keeps them real);
* volume sums over E points times dV; face sums over the face points times
  the transverse spacings;
* normal n from L (the -axis element) to R: [[u]] = u_L - u_R,
  {{d_n u}} = (d u_L + d u_R) / 2, which gives per face
      v,u in L:  -1/4 v du - 1/4 dv u + alpha v u
      v,u in R:  +1/4 v du + 1/4 dv u + alpha v u
      v in L, u in R:  -1/4 v du + 1/4 dv u - alpha v u   (and its transpose);
* alpha is used as given (Ha bohr); the nonlocal coupling of a pair of
  elements is put in the first stencil slot that names the pair, couplings
  to elements outside the stencil are dropped (their norm is reported);
* faces normal to an axis along which the element spans the whole periodic
  domain carry no jump and are skipped.

Block layout: blocks[k, s] has rows = test ALBs of element k and columns =
trial ALBs of element neighbors[k, s].
"""
from __future__ import annotations

import numpy as np

from .local_operator import projectors_on, v_local
from .alb import restrict

FACE_AXES = {1: 0, 3: 1, 5: 2, 7: 3, 9: 2}


def face_slot(axis, side):
    """Stencil slot of the face normal to `axis` on side -1 (low) or +1 (high)."""
    return 1 + 2 * axis + (0 if side < 0 else 1)


def spectral_derivative(F3, h, axis):
    """d/d(axis) of periodic grid functions F3 [n, Qz, Qy, Qx]; axis 0=x, 1=y, 2=z."""
    nv, nz, ny, nx = F3.shape
    n = (nx, ny, nz)[axis]
    m = np.fft.fftfreq(n) * n
    if n % 2 == 0:
        m[n // 2] = 0.0                      # Nyquist coefficient dropped
    G = 2.0 * np.pi * m / (n * h[axis])
    if axis == 0:
        G = G[: nx // 2 + 1]
        shape = (1, 1, 1, nx // 2 + 1)
    elif axis == 1:
        shape = (1, 1, ny, 1)
    else:
        shape = (1, nz, 1, 1)
    S = np.fft.rfftn(F3, axes=(1, 2, 3))
    return np.fft.irfftn(S * (1j * G.reshape(shape)), s=(nz, ny, nx), axes=(1, 2, 3))


def trace_weights(n, h, xf):
    """Weights w_val, w_der (length n) evaluating f(xf*h), f'(xf*h) of the trig interpolant of f_i = f(i h)."""
    i = np.arange(n)
    delta = (xf - i) * h
    mmax = (n - 1) // 2 if n % 2 else n // 2 - 1   # Nyquist dropped
    ms = np.arange(1, mmax + 1)
    G = 2.0 * np.pi * ms / (n * h)
    w_val = (1.0 + 2.0 * np.cos(G[None, :] * delta[:, None]).sum(1)) / n
    w_der = (-2.0 * (G[None, :] * np.sin(G[None, :] * delta[:, None])).sum(1)) / n
    return w_val, w_der


def face_traces(Psi3, prob, k, axis, side):
    """(val, der) [n_alb, F]: trace and normal derivative of Psi3 [n_alb, Qz, Qy, Qx] on a face of E_k."""
    dom = int(prob.elem_dom[k])
    h = prob.dom_h[dom]
    Qn = prob.elem_Qn[k]
    En = prob.elem_En[k]
    eo = (Qn - En) // 2
    xf = eo[axis] - 0.5 if side < 0 else eo[axis] + En[axis] - 0.5
    w_val, w_der = trace_weights(int(Qn[axis]), h[axis], xf)
    # restrict the transverse axes to E, keep the full normal line
    sl = [slice(None)] * 4
    for a in range(3):
        if a != axis:
            sl[3 - a] = slice(int(eo[a]), int(eo[a] + En[a]))
    P = Psi3[tuple(sl)]
    ax = 3 - axis
    val = np.tensordot(P, w_val, axes=([ax], [0]))
    der = np.tensordot(P, w_der, axes=([ax], [0]))
    return val.reshape(P.shape[0], -1), der.reshape(P.shape[0], -1)


def face_area(prob, k, axis):
    h = prob.dom_h[int(prob.elem_dom[k])]
    return float(np.prod([h[a] for a in range(3) if a != axis]))


def face_axes(prob, k):
    """Axes with real faces: those the stencil names and along which E_k does not span the domain."""
    dom = int(prob.elem_dom[k])
    return [a for a in range(FACE_AXES[prob.n_stencil])
            if int(prob.elem_En[k][a]) < int(prob.dom_n[dom][a])]


def element_ingredients(prob, k, X_eig, C, A):
    """Per-element DG ingredients from the eigenvectors X_eig [n_eig, N_Q], C [n_eig, n_alb], A [n_alb, N_E]."""
    dom = int(prob.elem_dom[k])
    h = prob.dom_h[dom]
    dV = float(np.prod(h))
    Qn = prob.elem_Qn[k]
    En = prob.elem_En[k]
    eo = (Qn - En) // 2
    Psi = C.T @ X_eig                                  # ALB extended to Q as trig interpolant
    Psi3 = Psi.reshape(Psi.shape[0], int(Qn[2]), int(Qn[1]), int(Qn[0]))
    kin = np.zeros((A.shape[0], A.shape[0]))
    for axis in range(3):
        D = restrict(spectral_derivative(Psi3, h, axis).reshape(Psi.shape[0], -1), Qn, eo, En)
        kin += 0.5 * (D @ D.T) * dV
    VE = restrict(v_local(prob, k).reshape(1, -1), Qn, eo, En)[0]
    vmat = (A * VE[None, :]) @ A.T * dV
    # projector overlaps P_{I,l,k} = <b_{I,l}|_E, A> dV
    gE = [np.mod(prob.elem_E0[k][a] + np.arange(int(En[a])), prob.dom_n[dom][a]) for a in range(3)]
    BE, gam, ids = projectors_on(prob, dom, gE[0], gE[1], gE[2])
    P = (BE.T @ A.T) * dV if BE.shape[1] else np.zeros((0, A.shape[0]))
    faces = {}
    for axis in face_axes(prob, k):
        for side in (-1, 1):
            faces[(axis, side)] = face_traces(Psi3, prob, k, axis, side)
    return dict(kin=kin, vmat=vmat, P=P, gamma=gam, ids=ids, faces=faces,
                n_alb=A.shape[0])


def nonlocal_block(ia, ib):
    """sum_{I,l} gamma <phi_a, b><b, phi_b> over projectors present in both elements."""
    out = np.zeros((ia["n_alb"], ib["n_alb"]))
    pos_b = {pid: r for r, pid in enumerate(ib["ids"])}
    for r, pid in enumerate(ia["ids"]):
        rb = pos_b.get(pid)
        if rb is not None:
            out += ia["gamma"][r] * np.outer(ia["P"][r], ib["P"][rb])
    return out


def diagonal_block(prob, k, ik, alpha):
    """H^DG_kk: kinetic + V_eff + nonlocal + the face terms with test and trial both in E_k."""
    B0 = ik["kin"] + ik["vmat"] + nonlocal_block(ik, ik)
    for (axis, side), (val, der) in ik["faces"].items():
        dA = face_area(prob, k, axis)
        sgn = 1.0 if side < 0 else -1.0   # k is R on its low face, L on its high face
        B0 = B0 + dA * (sgn * 0.25 * (val @ der.T + der @ val.T) + alpha * (val @ val.T))
    return B0


def assemble(prob, ingr, alpha):
    """DG blocks [M, n_stencil, max n_alb, max n_alb] (zero padded) and the dropped nonlocal norm."""
    M = prob.n_elem
    S = prob.n_stencil
    nmax = max(i["n_alb"] for i in ingr)
    blocks = np.zeros((M, S, nmax, nmax))
    for k in range(M):
        ik = ingr[k]
        nk = ik["n_alb"]
        blocks[k, 0, :nk, :nk] = diagonal_block(prob, k, ik, alpha)
        seen = {k}
        for s in range(1, S):
            kp = int(prob.neighbors[k, s])
            if kp < 0:
                continue
            ip = ingr[kp]
            npp = ip["n_alb"]
            blk = np.zeros((nk, npp))
            if s <= 2 * FACE_AXES[S]:
                axis = (s - 1) // 2
                side = -1 if (s - 1) % 2 == 0 else 1
                if (axis, side) in ik["faces"]:
                    dA = face_area(prob, k, axis)
                    vk, dk = ik["faces"][(axis, side)]
                    vp, dp = ip["faces"][(axis, -side)]
                    if side > 0:   # k = L, neighbour = R
                        blk += dA * (-0.25 * vk @ dp.T + 0.25 * dk @ vp.T - alpha * vk @ vp.T)
                    else:          # k = R, neighbour = L
                        blk += dA * (0.25 * vk @ dp.T - 0.25 * dk @ vp.T - alpha * vk @ vp.T)
            if kp not in seen:
                blk += nonlocal_block(ik, ip)
                seen.add(kp)
            blocks[k, s, :nk, :npp] = blk
    # norm of the nonlocal couplings to elements outside the stencil
    dropped = 0.0
    for k in range(M):
        inside = set(int(v) for v in prob.neighbors[k] if v >= 0)
        for kp in range(M):
            if kp not in inside and int(prob.elem_dom[kp]) == int(prob.elem_dom[k]):
                dropped += float(np.sum(nonlocal_block(ingr[k], ingr[kp]) ** 2))
    return blocks, float(np.sqrt(dropped))


def dense(prob, blocks, n_alb):
    """Dense H^DG (N_b x N_b) from the stencil blocks (Eq. DGEigenvalue)."""
    n_alb = np.asarray(n_alb, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(n_alb)])
    H = np.zeros((off[-1], off[-1]))
    for k in range(prob.n_elem):
        for s in range(prob.n_stencil):
            kp = int(prob.neighbors[k, s])
            if kp < 0:
                continue
            H[off[k]:off[k + 1], off[kp]:off[kp + 1]] += blocks[k, s, :n_alb[k], :n_alb[kp]]
    return H
