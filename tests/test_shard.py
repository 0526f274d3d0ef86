"""Element sharding (Sec. II.B: elements distributed among processes, neighbour data exchanged point to
point for H^DG) on two gloo ranks on the CPU.

The product's host logic in paper_2003_00407_gb300/shard.py -- tile partition, the exchange plan, the
packing and placement of records at the library's record offsets (dgdft_dg_query_layout, host only),
the point-to-point exchange and the gradient all-reduce -- runs unchanged; the per-element arithmetic
comes from the oracle through an adapter that writes its DG ingredients in the library's record layout
(the CUDA library needs a GPU; the same flow on the GPU is tests/test_gpu_shard.py).  The sharded DG
blocks and gradients must equal the single-process oracle result.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import driver, dg as odg
from oracle.local_operator import projectors_on
from workloads.configs import make_slab
from paper_2003_00407_gb300 import shard

ALPHA = 20.0
KT = 0.01


def small_slab(stencil=5):
    w = make_slab(4, 2, (8, 6, 12), (16, 12, 12), 0.45, 10, 6, 5, r_cut=2.6, width=0.7, proj_width=0.7,
                  stencil=stencil)
    w.alpha = ALPHA
    return w


class OracleBackend:
    """The oracle's per-element DG arithmetic behind the backend interface of shard.py, with the
    ingredients written in the library's record layout (test adapter)."""
    xp = np

    def __init__(self):
        from paper_2003_00407_gb300 import api, build
        build.build()
        self.api = api

    def layout(self, wl):
        return self.api.dg_layout(wl.problem, wl.params)

    def _L(self, wl):
        return int(np.max(wl.params.n_blk))

    def ingredients(self, wl, sols):
        p, q = wl.problem, wl.params
        tr_off, pe_off = self.layout(wl)
        M, L = p.n_elem, self._L(wl)
        kv = np.zeros((M, L, L))
        tr = np.zeros(max(1, int(tr_off[-1])))
        pe = np.zeros(max(1, int(pe_off[-1])))
        for k in range(M):
            s = sols[k]
            ik = odg.element_ingredients(p, k, s["X"][:s["n_eig"]], s["C"], s["A"])
            na = ik["n_alb"]
            kv[k, :na, :na] = ik["kin"] + ik["vmat"]
            flen = int(tr_off[k + 1] - tr_off[k]) // 6
            F = flen // (2 * na) if flen else 0
            for (axis, side), (val, der) in ik["faces"].items():
                f = 2 * axis + (1 if side > 0 else 0)
                rec = tr[tr_off[k] + f * flen: tr_off[k] + (f + 1) * flen].reshape(2, na, F)
                rec[0, :, :val.shape[1]] = val
                rec[1, :, :der.shape[1]] = der
            npk = ik["P"].shape[0]
            assert npk * na == int(pe_off[k + 1] - pe_off[k])
            pe[pe_off[k]:pe_off[k + 1]] = ik["P"].T.ravel()
        return kv, tr, pe

    def blocks(self, wl, kv, tr, pe, alpha):
        p, q = wl.problem, wl.params
        tr_off, pe_off = self.layout(wl)
        ingr = []
        for k in range(p.n_elem):
            na = int(q.n_alb[k])
            dom = int(p.elem_dom[k])
            gE = [np.mod(p.elem_E0[k][a] + np.arange(int(p.elem_En[k][a])), p.dom_n[dom][a]) for a in range(3)]
            _, gam, ids = projectors_on(p, dom, gE[0], gE[1], gE[2])
            flen = int(tr_off[k + 1] - tr_off[k]) // 6
            F = flen // (2 * na) if flen else 0
            faces = {}
            for axis in odg.face_axes(p, k):
                Fa = int(np.prod(p.elem_En[k])) // int(p.elem_En[k][axis])
                for side in (-1, 1):
                    f = 2 * axis + (1 if side > 0 else 0)
                    rec = tr[tr_off[k] + f * flen: tr_off[k] + (f + 1) * flen].reshape(2, na, F)
                    faces[(axis, side)] = (rec[0, :, :Fa], rec[1, :, :Fa])
            P = pe[pe_off[k]:pe_off[k + 1]].reshape(na, -1).T if na else np.zeros((0, 0))
            ingr.append(dict(kin=kv[k, :na, :na], vmat=np.zeros((na, na)), P=P, gamma=np.asarray(gam), ids=ids,
                             faces=faces, n_alb=na))
        blocks, _ = odg.assemble(p, ingr, alpha)
        return blocks

    def grad(self, wl, sols, kT, nel):
        return driver.alb_grad(wl.problem, sols, kT, nel)


def solve_all(wl, elems=None):
    elems = range(wl.problem.n_elem) if elems is None else elems
    return {int(k): driver.solve_element(wl.problem, wl.params, int(k), tol=1e-10, max_iter=300) for k in elems}


class NumpyComm:
    """shard.TorchComm over CPU tensors, converting to numpy for the oracle adapter."""

    def __init__(self, tc):
        self.tc, self.rank, self.world = tc, tc.rank, tc.world

    def exchange(self, sends, sizes):
        out = self.tc.exchange({q: torch.from_numpy(np.ascontiguousarray(v)) for q, v in sends.items()}, sizes)
        return {q: v.numpy() for q, v in out.items()}

    def allreduce(self, a):
        return self.tc.allreduce(torch.from_numpy(np.ascontiguousarray(a))).numpy()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, stencil, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ[v] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = small_slab(stencil)
        sh = shard.Shard(wl, world, rank)
        comm = NumpyComm(shard.TorchComm(dist, torch.device("cpu")))
        full = solve_all(wl, sh.local)
        local_sols = {i: full[int(k)] for i, k in enumerate(sh.local)}
        be = OracleBackend()
        blocks = shard.sharded_dg_blocks(sh, comm, be, local_sols)
        nel = np.full(wl.problem.n_elem, 4.0)      # two occupied states of the ten
        E, gv, gR = shard.sharded_grad(sh, comm, be, local_sols, KT, nel)
        out[rank] = dict(local=sh.local.tolist(), blocks=np.asarray(blocks), E=np.asarray(E), gv=np.asarray(gv),
                         gR=np.asarray(gR), peers=sh.peers)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("stencil", [5, 9])
def test_two_ranks_reproduce_the_single_process_blocks_and_gradient(stencil):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, stencil, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    wl = small_slab(stencil)
    sols = solve_all(wl)
    ref_blocks = driver.dg_assemble(wl.problem, sols, ALPHA)[0]
    nel = np.full(wl.problem.n_elem, 4.0)
    E_ref, gv_ref, gR_ref = driver.alb_grad(wl.problem, sols, KT, nel)
    seen = []
    for r in range(world):
        d = res[r]
        assert d["peers"] == [1 - r]
        loc = d["local"]
        seen += loc
        nmax = ref_blocks.shape[2]
        got = d["blocks"][:, :, :nmax, :nmax]
        err = np.abs(got - ref_blocks[loc]).max()
        assert err <= 1e-12 * max(1.0, np.abs(ref_blocks).max()), (r, err)
        assert np.abs(d["E"] - E_ref[loc]).max() <= 1e-12
        assert np.abs(d["gv"] - gv_ref).max() <= 1e-12 * max(1.0, np.abs(gv_ref).max())
        assert np.abs(d["gR"] - gR_ref).max() <= 1e-12 * max(1.0, np.abs(gR_ref).max())
    assert sorted(seen) == list(range(wl.problem.n_elem))


def test_partition_tiles_and_exchange_plan_agree():
    from workloads import make_config
    p = make_config(5).problem          # 32 x 32 element sheet
    for world in (1, 2, 4, 8):
        owner = shard.partition(p, world)
        assert sorted(set(owner.tolist())) == list(range(world))
        counts = np.bincount(owner, minlength=world)
        assert counts.min() == counts.max() == 1024 // world
        g = shard.element_grid(p)
        nex, ney, ex, ey = g
        for r in range(world):
            sel = owner == r
            # a tile is a full rectangle of the element grid
            bx, by = ex[sel], ey[sel]
            assert sel.sum() == (bx.max() - bx.min() + 1) * (by.max() - by.min() + 1)
        for r in range(world):
            for q in range(world):
                if r == q:
                    continue
                fs = shard.face_sends(p, owner, r, q)
                # every face sent is the face across which an element of q sees an element of r
                for k, f in fs:
                    n = int(p.neighbors[k, f + 1])
                    assert owner[n] == q and int(p.neighbors[n, (f ^ 1) + 1]) == k
    # independent elements (no single grid) split into contiguous id ranges
    c3 = make_config(3).problem
    owner = shard.partition(c3, 4)
    assert np.all(np.diff(owner) >= 0) and np.bincount(owner).tolist() == [64] * 4
