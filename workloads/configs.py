"""The five benchmark workloads and small test variants.

All draws use NumPy's PCG64 with ``seed = 20030407 + config index`` unless a
seed is given.  The graphene-like slabs mimic the paper's test systems (Sec.
III, graphene G180/G2880/G11520 partitioned in a 2D mesh along x and y):
isotropic spacing h = 0.4 bohr (E_cut = (pi/h)^2/2 ~ 30.8 Ha through
(N_r)_i = sqrt(2 E_cut) L_i / pi), 6.4 x 6.4 bohr elements with four atoms each
on a jittered 2x2 lattice, Gaussian local wells (depth U[2,4] Ha, sigma 0.8
bohr) and four Gaussian-radial Kleinman-Bylander projectors per atom
(gamma ~ U[0.5, 2.0] Ha, sigma 0.8 bohr), support radius 3.2 bohr.
"""
from __future__ import annotations

import math
import numpy as np

from .problem import (Problem, Params, Workload, STENCIL_SELF, STENCIL_XY,
                      STENCIL_XY9)

CONFIG_NAMES = {
    1: "c1-single-cube-16^3",
    2: "c2-slab-8x8-elem-32x32x48",
    3: "c3-uneven-256-elem",
    4: "c4-grad-8x8-elem-32x32x48",
    5: "c5-sheet-32x32-elem-32x32x48",
}

BASE_SEED = 20030407


def n_blk_rule(n_eig: int) -> int:
    """Filter block: n_eig plus max(4, ceil(n_eig/10)) guard vectors, rounded up to 8."""
    g = max(4, int(math.ceil(n_eig / 10.0)))
    return int(8 * math.ceil((n_eig + g) / 8.0))


def _params(n_eig, n_alb, M, degree=10, tol=1e-8, max_iter=60, seed=BASE_SEED):
    n_eig = np.broadcast_to(np.asarray(n_eig, dtype=np.int32), (M,)).copy()
    n_alb = np.broadcast_to(np.asarray(n_alb, dtype=np.int32), (M,)).copy()
    n_blk = np.array([n_blk_rule(int(v)) for v in n_eig], dtype=np.int32)
    return Params(n_eig=n_eig, n_alb=n_alb, n_blk=n_blk, cheb_degree=degree, tol=tol,
                  max_iter=max_iter, seed=seed)


def _neighbors_2d(nex, ney, stencil):
    """Periodic element mesh in x,y; element id = ey*nex + ex."""
    M = nex * ney
    nb = np.zeros((M, stencil), dtype=np.int32)
    for ey in range(ney):
        for ex in range(nex):
            k = ey * nex + ex
            idx = lambda dx, dy: ((ey + dy) % ney) * nex + (ex + dx) % nex
            row = [k, idx(-1, 0), idx(1, 0), idx(0, -1), idx(0, 1)]
            if stencil == STENCIL_XY9:
                row += [idx(-1, -1), idx(1, -1), idx(-1, 1), idx(1, 1)]
            nb[k, :] = row[:stencil]
    return nb


def make_slab(nex, ney, En, Qn, h, n_eig, n_alb, seed, *, n_proj=4, stencil=STENCIL_XY,
              jitter=0.4, zjitter=0.1, depth=(2.0, 4.0), width=0.8, gamma=(0.5, 2.0),
              proj_width=0.8, r_cut=3.2, lattice=2, degree=10, tol=1e-8, max_iter=60,
              name="slab", atoms_z_centre=True):
    """Graphene-like slab: nex x ney elements of En points, one periodic domain."""
    rng = np.random.Generator(np.random.PCG64(seed))
    En = np.asarray(En, dtype=np.int32)
    Qn = np.asarray(Qn, dtype=np.int32)
    n = np.array([nex * En[0], ney * En[1], En[2]], dtype=np.int32)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)).copy()
    L = n * h
    M = nex * ney
    E0 = np.zeros((M, 3), dtype=np.int32)
    for ey in range(ney):
        for ex in range(nex):
            E0[ey * nex + ex] = (ex * En[0], ey * En[1], 0)
    pos = []
    for k in range(M):
        base = E0[k] * h
        ext = En * h
        for ly in range(lattice):
            for lx in range(lattice):
                p = np.array([base[0] + (lx + 0.5) * ext[0] / lattice,
                              base[1] + (ly + 0.5) * ext[1] / lattice,
                              L[2] / 2.0 if atoms_z_centre else base[2] + ext[2] / 2.0])
                p[0] += rng.uniform(-jitter, jitter)
                p[1] += rng.uniform(-jitter, jitter)
                p[2] += rng.uniform(-zjitter, zjitter)
                pos.append(np.mod(p, L))
    pos = np.array(pos, dtype=np.float64)
    na = pos.shape[0]
    prob = Problem(
        dom_n=n[None, :].copy(), dom_h=h[None, :].copy(), dom_voff=np.zeros(1, dtype=np.int64),
        v_extra=np.zeros(int(np.prod(n)), dtype=np.float64),
        elem_dom=np.zeros(M, dtype=np.int32), elem_E0=E0,
        elem_En=np.tile(En, (M, 1)).astype(np.int32), elem_Qn=np.tile(Qn, (M, 1)).astype(np.int32),
        neighbors=_neighbors_2d(nex, ney, stencil), n_stencil=stencil,
        atom_dom=np.zeros(na, dtype=np.int32), atom_pos=pos,
        well_depth=rng.uniform(depth[0], depth[1], na),
        well_width=np.full(na, width),
        n_proj_per_atom=n_proj,
        proj_gamma=rng.uniform(gamma[0], gamma[1], (na, n_proj)) if n_proj else np.zeros((na, 0)),
        proj_width=np.full(na, proj_width),
        r_cut=float(r_cut))
    params = _params(n_eig, n_alb, M, degree=degree, tol=tol, max_iter=max_iter, seed=seed)
    n_el = electrons_per_element(prob)
    return Workload(name=name, problem=prob, params=params, n_electrons=n_el)


def electrons_per_element(prob: Problem, per_atom: int = 4) -> np.ndarray:
    """4 valence electrons (carbon-like) for each atom whose nearest grid point lies in E_k."""
    M = prob.n_elem
    out = np.zeros(M, dtype=np.float64)
    for k in range(M):
        d = int(prob.elem_dom[k])
        sel = prob.atom_dom == d
        if not np.any(sel):
            continue
        h = prob.dom_h[d]
        n = prob.dom_n[d]
        idx = np.floor(prob.atom_pos[sel] / h + 0.5).astype(np.int64) % n
        rel = (idx - prob.elem_E0[k]) % n
        out[k] = per_atom * np.count_nonzero(np.all(rel < prob.elem_En[k], axis=1))
    return out


def make_cube(seed, n=16, L=10.0, n_wells=8, n_eig=16, n_alb=8, En=8, n_proj=0,
              degree=10, tol=1e-8, max_iter=60, name="cube"):
    """One periodic cube; Q is the whole box, E its central En^3 block."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = L / n
    pos = rng.uniform(0.0, L, (n_wells, 3))
    nn = np.array([n, n, n], dtype=np.int32)
    E0 = (n - En) // 2
    prob = Problem(
        dom_n=nn[None, :].copy(), dom_h=np.full((1, 3), h), dom_voff=np.zeros(1, dtype=np.int64),
        v_extra=np.zeros(n ** 3), elem_dom=np.zeros(1, dtype=np.int32),
        elem_E0=np.array([[E0, E0, E0]], dtype=np.int32),
        elem_En=np.array([[En, En, En]], dtype=np.int32),
        elem_Qn=np.array([[n, n, n]], dtype=np.int32),
        neighbors=np.zeros((1, 1), dtype=np.int32), n_stencil=STENCIL_SELF,
        atom_dom=np.zeros(n_wells, dtype=np.int32), atom_pos=pos,
        well_depth=rng.uniform(2.0, 4.0, n_wells), well_width=np.full(n_wells, 0.8),
        n_proj_per_atom=n_proj,
        proj_gamma=rng.uniform(0.5, 2.0, (n_wells, n_proj)) if n_proj else np.zeros((n_wells, 0)),
        proj_width=np.full(n_wells, 0.8), r_cut=3.2)
    params = _params(n_eig, n_alb, 1, degree=degree, tol=tol, max_iter=max_iter, seed=seed)
    return Workload(name=name, problem=prob, params=params,
                    n_electrons=np.array([8.0]))


def make_uneven(n_elem, seed, *, sizes_xy=(24, 32, 40), sizes_z=(32, 48), h=0.4,
                atoms=(2, 6), n_alb=(20, 60), degree=10, tol=1e-8, max_iter=60,
                name="uneven"):
    """Independent elements, each its own periodic domain equal to Q.

    E is the central half of Q in x and y and all of Q in z.  Atoms sit at
    uniform random x,y inside E, z at the slab centre +-0.1 bohr.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dom_n, dom_voff, E0s, Ens, Qns = [], [], [], [], []
    apos, adom, n_alb_l = [], [], []
    off = 0
    for k in range(n_elem):
        q = np.array([rng.choice(sizes_xy), rng.choice(sizes_xy), rng.choice(sizes_z)], dtype=np.int32)
        e = np.array([q[0] // 2, q[1] // 2, q[2]], dtype=np.int32)
        e0 = (q - e) // 2
        dom_n.append(q); dom_voff.append(off); off += int(np.prod(q))
        E0s.append(e0); Ens.append(e); Qns.append(q)
        na = int(rng.integers(atoms[0], atoms[1] + 1))
        for _ in range(na):
            p = np.array([(e0[0] + rng.uniform(0, e[0])) * h, (e0[1] + rng.uniform(0, e[1])) * h,
                          q[2] * h / 2.0 + rng.uniform(-0.1, 0.1)])
            apos.append(p); adom.append(k)
        n_alb_l.append(int(rng.integers(n_alb[0], n_alb[1] + 1)))
    na = len(apos)
    n_alb_a = np.array(n_alb_l, dtype=np.int32)
    n_eig_a = np.ceil(1.25 * n_alb_a).astype(np.int32)
    prob = Problem(
        dom_n=np.array(dom_n, dtype=np.int32), dom_h=np.full((n_elem, 3), h),
        dom_voff=np.array(dom_voff, dtype=np.int64), v_extra=np.zeros(off),
        elem_dom=np.arange(n_elem, dtype=np.int32), elem_E0=np.array(E0s, dtype=np.int32),
        elem_En=np.array(Ens, dtype=np.int32), elem_Qn=np.array(Qns, dtype=np.int32),
        neighbors=np.arange(n_elem, dtype=np.int32)[:, None].copy(), n_stencil=STENCIL_SELF,
        atom_dom=np.array(adom, dtype=np.int32), atom_pos=np.array(apos, dtype=np.float64),
        well_depth=rng.uniform(2.0, 4.0, na), well_width=np.full(na, 0.8), n_proj_per_atom=4,
        proj_gamma=rng.uniform(0.5, 2.0, (na, 4)), proj_width=np.full(na, 0.8), r_cut=3.2)
    params = _params(n_eig_a, n_alb_a, n_elem, degree=degree, tol=tol, max_iter=max_iter, seed=seed)
    wl = Workload(name=name, problem=prob, params=params)
    wl.n_electrons = electrons_per_element(prob)
    return wl


def make_config(k: int, seed: int | None = None, **kw) -> Workload:
    """Workload for benchmark configuration k (1..5)."""
    s = BASE_SEED + k if seed is None else seed
    if k == 1:
        wl = make_cube(s, **kw)
        wl.description = ("periodic 10 bohr cube, 16^3 grid, 8 Gaussian wells, no projectors; "
                          "16 eigenpairs (block 24), degree 10, tol 1e-8; central 8^3 element, 8 ALBs")
    elif k == 2:
        wl = make_slab(8, 8, (16, 16, 48), (32, 32, 48), 0.4, 40, 32, s, name=CONFIG_NAMES[2], **kw)
        wl.description = ("8x8 elements of 16x16x48 (Q 32x32x48, h 0.4), 4 atoms/element with wells "
                          "and 4 KB projectors; 40 eigenpairs (block 48), 32 ALBs; alpha 20")
    elif k == 3:
        wl = make_uneven(256, s, name=CONFIG_NAMES[3], **kw)
        wl.description = ("256 independent elements, Q from {24,32,40}^2 x {32,48}, 2-6 atoms, "
                          "20-60 ALBs, n_eig = ceil(1.25 n_alb)")
    elif k == 4:
        # 48 eigenpairs: with 40 the highest one is not empty enough (f >= 1e-12) on some elements
        wl = make_slab(8, 8, (16, 16, 48), (32, 32, 48), 0.4, 48, 32, s, name=CONFIG_NAMES[4], **kw)
        wl.kT = 0.01
        wl.description = ("config-2 geometry, 48 eigenpairs (block 56); Fermi smearing kT 0.01 Ha; "
                          "gradient w.r.t. V_eff and atoms")
    elif k == 5:
        wl = make_slab(32, 32, (16, 16, 48), (32, 32, 48), 0.4, 72, 64, s, name=CONFIG_NAMES[5], **kw)
        wl.description = ("32x32 elements of 16x16x48 (Q 32x32x48), 4096 atoms; 72 eigenpairs "
                          "(block 80), 64 ALBs; DG 64x64 blocks, 5-block stencil")
    else:
        raise ValueError(f"unknown config {k}")
    if k != 3:
        wl.name = CONFIG_NAMES[k]
    return wl


def subset(wl: Workload, elems) -> Workload:
    """Workload restricted to a subset of elements (for sampled oracle checks).

    Neighbour ids are kept as they are (they refer to the full partition); only
    element-local quantities may be computed from the subset.
    """
    import copy
    elems = np.asarray(elems, dtype=np.int64)
    p = copy.copy(wl.problem)
    p.elem_dom = p.elem_dom[elems].copy()
    p.elem_E0 = p.elem_E0[elems].copy()
    p.elem_En = p.elem_En[elems].copy()
    p.elem_Qn = p.elem_Qn[elems].copy()
    p.neighbors = p.neighbors[elems].copy()
    q = copy.copy(wl.params)
    q.n_eig = q.n_eig[elems].copy(); q.n_alb = q.n_alb[elems].copy(); q.n_blk = q.n_blk[elems].copy()
    out = copy.copy(wl)
    out.problem = p; out.params = q
    out.n_electrons = wl.n_electrons[elems].copy() if len(wl.n_electrons) else wl.n_electrons
    return out


def probe_directions(n: int, size: int, seed: int) -> np.ndarray:
    """n seeded random unit vectors of length size (to compare large gradients through projections)."""
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((n, size))
    return r / np.linalg.norm(r, axis=1, keepdims=True)


def probe_points(n: int, size: int, seed: int) -> np.ndarray:
    """n distinct seeded indices in [0, size)."""
    return np.sort(np.random.default_rng(seed).choice(size, size=n, replace=False))
