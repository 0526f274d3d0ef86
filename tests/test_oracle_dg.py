"""Pins of the DG assembly (Eq. DGHamiltonian, Eq. DGvar)."""
import numpy as np
import pytest

from oracle import dg, driver, local_operator as lo
from workloads.configs import make_slab, make_cube
from workloads.problem import STENCIL_XY9, STENCIL_XY


def test_spectral_derivative_exact_on_trig_polynomial():
    nx, ny, nz, h = 12, 10, 8, (0.5, 0.6, 0.7)
    L = (nx * h[0], ny * h[1], nz * h[2])
    x = np.arange(nx) * h[0]; y = np.arange(ny) * h[1]; z = np.arange(nz) * h[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    kx, ky, kz = 2 * np.pi * 2 / L[0], 2 * np.pi / L[1], 2 * np.pi * 3 / L[2]
    f = np.sin(kx * X) * np.cos(ky * Y) * np.cos(kz * Z)
    d = [dg.spectral_derivative(f[None], h, a)[0] for a in range(3)]
    np.testing.assert_allclose(d[0], kx * np.cos(kx * X) * np.cos(ky * Y) * np.cos(kz * Z), atol=1e-12)
    np.testing.assert_allclose(d[1], -ky * np.sin(kx * X) * np.sin(ky * Y) * np.cos(kz * Z), atol=1e-12)
    np.testing.assert_allclose(d[2], -kz * np.sin(kx * X) * np.cos(ky * Y) * np.sin(kz * Z), atol=1e-12)


def _brute_trace(f3, h, axis, pos_idx, eo, En):
    """Direct DFT evaluation of the trig interpolant (normal Nyquist dropped) on a face plane."""
    nz, ny, nx = f3.shape
    n = (nx, ny, nz)
    c = np.fft.fftn(f3) / f3.size                 # c[mz, my, mx]
    ms = [np.fft.fftfreq(m) * m for m in n]
    keep = np.ones(n[axis], dtype=bool)
    if n[axis] % 2 == 0:
        keep[n[axis] // 2] = False
    pts = []
    ranges = [np.arange(eo[a], eo[a] + En[a]) for a in range(3)]
    ranges[axis] = np.array([pos_idx])
    val, der = [], []
    for zz in ranges[2]:
        for yy in ranges[1]:
            for xx in ranges[0]:
                r = (xx * h[0], yy * h[1], zz * h[2])
                ph = np.exp(1j * (2 * np.pi * ms[2][:, None, None] * r[2] / (n[2] * h[2])
                                  + 2 * np.pi * ms[1][None, :, None] * r[1] / (n[1] * h[1])
                                  + 2 * np.pi * ms[0][None, None, :] * r[0] / (n[0] * h[0])))
                mask = np.ones_like(ph, dtype=bool)
                G = 2 * np.pi * ms[axis] / (n[axis] * h[axis])
                shape = [1, 1, 1]; shape[2 - axis] = n[axis]
                mask = mask & keep.reshape(shape)
                val.append(np.real((c * ph * mask).sum()))
                der.append(np.real((c * ph * mask * (1j * G.reshape(shape))).sum()))
    return np.array(val), np.array(der)


def test_face_traces_match_brute_force_dft():
    w = make_slab(2, 2, (6, 4, 5), (10, 8, 5), 0.45, 4, 2, 3)
    p = w.problem
    rng = np.random.default_rng(4)
    k = 1
    Qn = p.elem_Qn[k]
    f3 = rng.normal(size=(int(Qn[2]), int(Qn[1]), int(Qn[0])))
    eo = (Qn - p.elem_En[k]) // 2
    h = p.dom_h[0]
    for axis in (0, 1):
        for side in (-1, 1):
            val, der = dg.face_traces(f3[None], p, k, axis, side)
            pos = eo[axis] - 0.5 if side < 0 else eo[axis] + p.elem_En[k][axis] - 0.5
            bv, bd = _brute_trace(f3, h, axis, pos, eo, p.elem_En[k])
            np.testing.assert_allclose(val[0], bv, atol=1e-11)
            np.testing.assert_allclose(der[0], bd, atol=1e-10)


def _nyquist_deficit(X3, h, dV):
    """sum_a 1/2 (pi/h_a)^2 <psi_i^nyq,a, psi_j^nyq,a>: kinetic weight the spectral gradients drop."""
    nv = X3.shape[0]
    F = np.fft.fftn(X3, axes=(1, 2, 3))
    D = np.zeros((nv, nv))
    for a in range(3):
        na = X3.shape[3 - a]
        if na % 2:
            continue
        sl = [slice(None)] * 4
        sl[3 - a] = na // 2
        Fa = F[tuple(sl)].reshape(nv, -1)
        D += 0.5 * (np.pi / h[a]) ** 2 * np.real(Fa @ Fa.conj().T) * dV / X3[0].size
    return D


def _whole_box_2x2(n_eig, n_alb, seed=3, stencil=STENCIL_XY9):
    # 2x2 elements of 6x6x12 in a 12^3 box at h = 0.5; every Q is the whole box
    w = make_slab(2, 2, (6, 6, 12), (12, 12, 12), 0.5, n_eig, n_alb, seed, stencil=stencil,
                  width=0.7, proj_width=0.7, r_cut=2.8, lattice=1, jitter=0.3)
    return w


def _sols_dense(w):
    return {k: driver.solve_element(w.problem, w.params, k, dense_route=True)
            for k in range(w.problem.n_elem)}


def _ingredients(w, sols):
    return [dg.element_ingredients(w.problem, k, sols[k]["X"][:sols[k]["n_eig"]], sols[k]["C"],
                                   sols[k]["A"]) for k in range(w.problem.n_elem)]


def test_dg_quadratic_form_equals_energy_of_eq_dgvar():
    # c^T H^DG c against a direct evaluation of Eq. DGvar's terms for a discontinuous psi
    w = _whole_box_2x2(8, 6)
    p = w.problem
    sols = _sols_dense(w)
    ingr = _ingredients(w, sols)
    alpha = 7.0
    blocks, dropped = dg.assemble(p, ingr, alpha)
    H = dg.dense(p, blocks, w.params.n_alb)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    assert dropped == 0.0
    rng = np.random.default_rng(0)
    c = rng.normal(size=H.shape[0])
    off = np.concatenate([[0], np.cumsum(w.params.n_alb)])
    E = 0.0
    trace = {}
    for k in range(p.n_elem):
        ck = c[off[k]:off[k + 1]]
        ik = ingr[k]
        E += ck @ (ik["kin"] + ik["vmat"]) @ ck
        for (axis, side), (val, der) in ik["faces"].items():
            trace[(k, axis, side)] = (ck @ val, ck @ der)
    # nonlocal: sum_I,l gamma |<b, psi>|^2 with <b, psi> = sum_k P_k c_k
    proj = {}
    for k in range(p.n_elem):
        ck = c[off[k]:off[k + 1]]
        for r, pid in enumerate(ingr[k]["ids"]):
            proj[pid] = proj.get(pid, 0.0) + ingr[k]["P"][r] @ ck
            gam = ingr[k]["gamma"][r]
            proj[(pid, "g")] = gam
    E += sum(proj[(pid, "g")] * proj[pid] ** 2 for pid in list(proj) if not isinstance(pid[1], str))
    # faces: each face once, from its low (L) element's +side
    for k in range(p.n_elem):
        for axis in (0, 1):
            kr = int(p.neighbors[k, dg.face_slot(axis, +1)])
            vL, dL = trace[(k, axis, +1)]
            vR, dR = trace[(kr, axis, -1)]
            jump = vL - vR
            avg = 0.5 * (dL + dR)
            dA = dg.face_area(p, k, axis)
            E += (-(avg * jump).sum() + alpha * (jump * jump).sum()) * dA
    assert abs(c @ H @ c - E) < 1e-10 * abs(E)


def test_dg_reproduces_plane_wave_levels_for_continuous_functions():
    # Q = whole box: global eigenfunctions are continuous across faces, so face terms cancel
    # and the Galerkin form on them is diag(lambda)
    w = _whole_box_2x2(10, 10)
    p = w.problem
    sols = _sols_dense(w)
    blocks, _ = dg.assemble(p, _ingredients(w, sols), 20.0)
    H = dg.dense(p, blocks, w.params.n_alb)
    Q0 = lo.q_origin(p, 0)
    s0 = sols[0]
    n = p.dom_n[0]
    # global eigenvectors (from element 0's Q, shifted back to global indexing)
    Xg = np.roll(s0["X"][:6].reshape(6, *n[::-1]), shift=tuple(int(v) for v in Q0[::-1]), axis=(1, 2, 3))
    cs = []
    for j in range(6):
        parts = []
        for k in range(p.n_elem):
            gx, gy, gz = [np.mod(p.elem_E0[k][a] + np.arange(p.elem_En[k][a]), n[a]) for a in range(3)]
            psiE = Xg[j][np.ix_(gz, gy, gx)].ravel()
            parts.append(sols[k]["A"] @ psiE * s0["dV"])
        cs.append(np.concatenate(parts))
    Cm = np.array(cs)
    G = Cm @ H @ Cm.T
    np.testing.assert_allclose(Cm @ Cm.T, np.eye(6), atol=1e-9)
    # the DG kinetic term uses spectral gradients without the Nyquist coefficient while the
    # plane-wave kinetic keeps 1/2 G_nyq^2 on it: subtract exactly that deficit
    F = np.fft.fftn(Xg, axes=(1, 2, 3))
    h = p.dom_h[0]
    deficit = np.zeros((6, 6))
    for a in range(3):
        na = int(n[a]); gn = np.pi / h[a]
        sl = [slice(None)] * 4
        sl[3 - a] = na // 2
        Fa = F[tuple(sl)].reshape(6, -1)
        deficit += 0.5 * gn * gn * np.real(Fa @ Fa.conj().T) * s0["dV"] / Xg[0].size
    assert np.abs(deficit).max() > 1e-7          # the effect is real at this spacing
    np.testing.assert_allclose(G, np.diag(s0["theta"][:6]) - deficit, atol=1e-10)


def test_single_element_whole_box_equals_local_eigenvalues():
    w = make_cube(6, n=10, L=7.0, n_wells=3, n_proj=4, En=10, n_eig=8, n_alb=8)
    p = w.problem
    sols = _sols_dense(w)
    blocks, _ = dg.assemble(p, _ingredients(w, sols), 20.0)
    ev = np.linalg.eigvalsh(dg.dense(p, blocks, w.params.n_alb))
    # E = Q = whole box: H^DG is Lambda minus the Nyquist kinetic deficit, in an orthonormal basis
    X = sols[0]["X"][:8]
    D = _nyquist_deficit(X.reshape(8, 10, 10, 10), p.dom_h[0], sols[0]["dV"])
    ref = np.linalg.eigvalsh(np.diag(sols[0]["theta"][:8]) - D)
    np.testing.assert_allclose(ev, ref, atol=1e-10)
    # with projectors but a smooth enough grid the deficit is negligible
    assert np.abs(D).max() < 5e-3


@pytest.mark.slow
def test_dg_levels_monotone_in_nested_alb_spaces_and_near_plane_wave():
    # n_eig = n_alb gives nested ALB spaces (restrictions of the first n_eig eigenvectors), so by
    # min-max the DG levels cannot increase as n_alb grows; they approach the plane-wave levels
    # from below (the broken space is richer) to within 2e-3 Ha once n_alb >= 4.
    prev = None
    for n_alb in (2, 4, 8, 16, 32):
        w = _whole_box_2x2(n_alb, n_alb)
        p = w.problem
        sols = _sols_dense(w)
        blocks, _ = dg.assemble(p, _ingredients(w, sols), 20.0)
        ev = np.linalg.eigvalsh(dg.dense(p, blocks, w.params.n_alb))[:4]
        if prev is not None:
            assert np.all(ev <= prev + 1e-10), (n_alb, ev, prev)
        if n_alb >= 4:
            assert np.abs(ev - sols[0]["theta"][:4]).max() <= 2e-3
        prev = ev
