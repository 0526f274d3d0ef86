"""Element sharding across processes (Sec. II.B of the paper: the elements are distributed among the
processes, each process generates the ALBs of its own elements, and building H^DG needs the face and
projector data of neighbouring elements owned by other processes, exchanged point to point).

One process per GPU owns a contiguous 2D tile of the element grid.  Per process:

1. ALB generation (``api.alb_generate``) for its own elements only -- no communication;
2. DG ingredients (``api.dg_ingredients``) of its own elements;
3. one exchange: every element on the tile boundary sends, to each process owning one of its stencil
   neighbours, the face traces of the face shared with that neighbour and its projector overlaps;
4. DG blocks (``api.dg_blocks``) of its own elements from its records plus the received halo records;
5. for the band-energy gradient: each process forms the gradient of its own elements' energies, and the
   V_eff gradient (supported on the overlapping extended elements Q_k) and the atom gradient are summed
   over processes (an all-reduce, which is the halo add of the overlapping Q regions).

Host logic only: the arithmetic runs in the CUDA library through ``api``; communication goes through a
``comm`` object with ``rank``, ``world``, ``exchange(sends) -> recvs`` and ``allreduce(tensor)``
(``TorchComm`` wraps torch.distributed: gloo on CPU tensors, NCCL on CUDA tensors).
"""
from __future__ import annotations

import math

import numpy as np

FACE_AXES = {1: 0, 3: 1, 5: 2, 7: 3, 9: 2}


# ------------------------------------------------------------------ partition --
def element_grid(prob):
    """(nex, ney, ex, ey) when the elements tile one domain as a 2D grid along x and y, else None."""
    if len(set(int(d) for d in prob.elem_dom)) != 1:
        return None
    En = prob.elem_En
    if not (np.all(En == En[0])):
        return None
    ex = prob.elem_E0[:, 0] // En[0, 0]
    ey = prob.elem_E0[:, 1] // En[0, 1]
    nex, ney = int(ex.max()) + 1, int(ey.max()) + 1
    if nex * ney != prob.n_elem or len(set(zip(ex.tolist(), ey.tolist()))) != prob.n_elem:
        return None
    return nex, ney, ex.astype(np.int64), ey.astype(np.int64)


def tile_shape(world, nex, ney):
    """px x py = world process tiles, as square as the element grid allows."""
    best = None
    for px in range(1, world + 1):
        if world % px:
            continue
        py = world // px
        if px > nex or py > ney:
            continue
        cost = abs(math.log((nex / px) / (ney / py)))
        if best is None or cost < best[0]:
            best = (cost, px, py)
    return (best[1], best[2]) if best else (world, 1)


def partition(prob, world):
    """Owner rank of every element: contiguous 2D tiles of the element grid (contiguous id ranges when
    the elements do not form one grid, e.g. independent uneven elements)."""
    owner = np.zeros(prob.n_elem, dtype=np.int64)
    g = element_grid(prob)
    if g is None or world == 1:
        for r in range(world):
            owner[r * prob.n_elem // world:(r + 1) * prob.n_elem // world] = r
        return owner
    nex, ney, ex, ey = g
    px, py = tile_shape(world, nex, ney)
    tx = (ex * px) // nex
    ty = (ey * py) // ney
    return (ty * px + tx).astype(np.int64)


# ------------------------------------------------------------------ exchange plan --
def face_sends(prob, owner, src, dst):
    """Sorted (element, face) pairs that rank src sends to rank dst: faces of src's elements whose
    neighbour across the face is owned by dst (face = slot - 1 = 2*axis + high side)."""
    nf = 2 * FACE_AXES[int(prob.n_stencil)]
    out = []
    for k in np.nonzero(owner == src)[0]:
        for s in range(1, nf + 1):
            n = int(prob.neighbors[k, s])
            if n >= 0 and owner[n] == dst:
                out.append((int(k), s - 1))
    return sorted(set(out))


def proj_sends(prob, owner, src, dst):
    """Sorted elements of src with any stencil neighbour owned by dst (their projector overlaps enter the
    nonlocal coupling of the neighbour's blocks)."""
    out = set()
    for k in np.nonzero(owner == src)[0]:
        for s in range(1, int(prob.n_stencil)):
            n = int(prob.neighbors[k, s])
            if n >= 0 and owner[n] == dst:
                out.add(int(k))
    return sorted(out)


def sub_problem(wl, elems):
    """Workload restricted to `elems` (in that order), neighbours renumbered inside it (-1 outside)."""
    from workloads.configs import subset
    elems = np.asarray(elems, dtype=np.int64)
    w = subset(wl, elems)
    pos = {int(k): i for i, k in enumerate(elems)}
    nb = wl.problem.neighbors[elems]
    w.problem.neighbors = np.array([[pos.get(int(v), -1) if v >= 0 else -1 for v in row] for row in nb],
                                   dtype=np.int32).reshape(nb.shape)
    return w


class Shard:
    """The elements of one rank and the records it exchanges.

    local: owned elements (global ids, ascending); halo: elements of other ranks in their stencils;
    the block sub-problem lists local then halo elements."""

    def __init__(self, wl, world, rank):
        self.wl, self.world, self.rank = wl, world, rank
        p = wl.problem
        self.owner = partition(p, world)
        self.local = np.nonzero(self.owner == rank)[0]
        halo = set()
        for k in self.local:
            for s in range(1, int(p.n_stencil)):
                n = int(p.neighbors[k, s])
                if n >= 0 and self.owner[n] != rank:
                    halo.add(n)
        self.halo = np.array(sorted(halo), dtype=np.int64)
        self.order = np.concatenate([self.local, self.halo]).astype(np.int64)
        self.pos = {int(k): i for i, k in enumerate(self.order)}
        self.local_wl = sub_problem(wl, self.local)
        self.block_wl = sub_problem(wl, self.order)
        self.peers = sorted(set(int(self.owner[n]) for n in self.halo))

    # record geometry of an element (shared by all problems that contain it)
    def _face_len(self, tr_off, i, k):
        n_alb = int(self.wl.params.n_alb[k])
        rec = int(tr_off[i + 1] - tr_off[i])
        return rec // 6, n_alb                # one face: [2][n_alb][F] = rec / 6 scalars

    def pack(self, tr_local, pe_local, layout_local, dst):
        """Flat float64 array of what this rank sends to dst: the face records, then the overlap records."""
        tr_off, pe_off = layout_local
        lpos = {int(k): i for i, k in enumerate(self.local)}
        parts = []
        for k, f in face_sends(self.wl.problem, self.owner, self.rank, dst):
            i = lpos[k]
            flen, _ = self._face_len(tr_off, i, k)
            parts.append(tr_local[tr_off[i] + f * flen: tr_off[i] + (f + 1) * flen])
        for k in proj_sends(self.wl.problem, self.owner, self.rank, dst):
            i = lpos[k]
            parts.append(pe_local[pe_off[i]:pe_off[i + 1]])
        return parts

    def recv_sizes(self, layout_block, src):
        """Sizes (scalars) of the face and overlap records this rank receives from src."""
        tr_off, pe_off = layout_block
        sizes = []
        for k, f in face_sends(self.wl.problem, self.owner, src, self.rank):
            i = self.pos[k]
            sizes.append(int(tr_off[i + 1] - tr_off[i]) // 6)
        for k in proj_sends(self.wl.problem, self.owner, src, self.rank):
            i = self.pos[k]
            sizes.append(int(pe_off[i + 1] - pe_off[i]))
        return sizes

    def place(self, xp, tr_block, pe_block, layout_block, src, flat):
        """Writes the records received from src (one flat array) into the block sub-problem's arrays."""
        tr_off, pe_off = layout_block
        o = 0
        for k, f in face_sends(self.wl.problem, self.owner, src, self.rank):
            i = self.pos[k]
            flen = int(tr_off[i + 1] - tr_off[i]) // 6
            tr_block[tr_off[i] + f * flen: tr_off[i] + (f + 1) * flen] = flat[o:o + flen]
            o += flen
        for k in proj_sends(self.wl.problem, self.owner, src, self.rank):
            i = self.pos[k]
            n = int(pe_off[i + 1] - pe_off[i])
            pe_block[pe_off[i]:pe_off[i] + n] = flat[o:o + n]
            o += n
        assert o == len(flat), (o, len(flat))


def _zeros_like(xp, ref, n):
    if hasattr(xp, "cuda"):          # torch
        return xp.zeros(n, dtype=ref.dtype, device=ref.device)
    return np.zeros(n)


def _cat(xp, parts, ref):
    if not parts:
        return _zeros_like(xp, ref, 0)
    return xp.cat(parts) if hasattr(xp, "cat") else np.concatenate(parts)


def dg_prepare(shard, backend, res_local):
    """Step 2 and the send side of step 3: the local ingredients and, per peer rank, the flat array of
    records to send.  Returns a state for dg_finish."""
    kv, tr, pe = backend.ingredients(shard.local_wl, res_local)
    lay_l = backend.layout(shard.local_wl)
    lay_b = backend.layout(shard.block_wl)
    sends = {q: _cat(backend.xp, shard.pack(tr, pe, lay_l, q), tr) for q in shard.peers}
    sizes = {q: sum(shard.recv_sizes(lay_b, q)) for q in shard.peers}
    return dict(kv=kv, tr=tr, pe=pe, lay_l=lay_l, lay_b=lay_b, sends=sends, sizes=sizes)


def dg_finish(shard, backend, st, recvs):
    """Receive side of step 3 and step 4: the block sub-problem's ingredient arrays (own records copied,
    halo records placed) and the DG blocks [n_local, n_stencil, L, L] of the local elements."""
    xp = backend.xp
    kv_l, tr_l, pe_l = st["kv"], st["tr"], st["pe"]
    (tr_off_l, pe_off_l), (tr_off_b, pe_off_b) = st["lay_l"], st["lay_b"]
    nl = len(shard.local)
    tr_b = _zeros_like(xp, tr_l, max(1, int(tr_off_b[-1])))
    pe_b = _zeros_like(xp, pe_l, max(1, int(pe_off_b[-1])))
    # own records are the first nl elements of the block sub-problem, in the same order
    assert int(tr_off_b[nl]) == int(tr_off_l[nl]) and int(pe_off_b[nl]) == int(pe_off_l[nl])
    tr_b[:int(tr_off_l[nl])] = tr_l[:int(tr_off_l[nl])]
    pe_b[:int(pe_off_l[nl])] = pe_l[:int(pe_off_l[nl])]
    for q in shard.peers:
        shard.place(xp, tr_b, pe_b, st["lay_b"], q, recvs[q])
    L = int(kv_l.shape[1])
    nb = len(shard.order)
    kv_b = _zeros_like(xp, kv_l, nb * L * L).reshape(nb, L, L)
    kv_b[:nl] = kv_l
    blocks = backend.blocks(shard.block_wl, kv_b, tr_b, pe_b, shard.wl.alpha)
    return blocks[:nl]


# ------------------------------------------------------------------ comms --
class TorchComm:
    """Point-to-point exchange and all-reduce over torch.distributed (gloo: CPU tensors, NCCL: CUDA)."""

    def __init__(self, dist, device):
        self.dist, self.device = dist, device
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    def exchange(self, sends, sizes):
        import torch
        reqs, recvs = [], {}
        for q in sorted(set(sends) | set(sizes)):
            recvs[q] = torch.empty(int(sizes.get(q, 0)), dtype=torch.float64, device=self.device)
            if q in sends and sends[q].numel():
                reqs.append(self.dist.isend(torch.as_tensor(sends[q]).to(self.device).contiguous(), q))
            if recvs[q].numel():
                reqs.append(self.dist.irecv(recvs[q], q))
        for r in reqs:
            r.wait()
        return recvs

    def allreduce(self, t):
        import torch
        tt = torch.as_tensor(t).to(self.device)
        self.dist.all_reduce(tt)
        return tt


def sharded_dg_blocks(shard, comm, backend, res_local):
    """DG blocks [n_local, n_stencil, L, L] of this rank's elements (steps 2-4 above).

    backend provides ingredients(wl, res) -> (kv, traces, proj), blocks(wl, kv, traces, proj, alpha),
    layout(wl) -> (tr_off, pe_off) and xp (the array module of its arrays)."""
    st = dg_prepare(shard, backend, res_local)
    recvs = comm.exchange(st["sends"], st["sizes"])
    return dg_finish(shard, backend, st, recvs)


def sharded_grad(shard, comm, backend, res_local, kT, n_electrons):
    """(energies of the local elements, V_eff gradient on the global grid, atom gradient): the local
    elements' contributions, with the two gradients summed over all ranks.  n_electrons: [M] of the whole
    partition."""
    nel = np.asarray(n_electrons, dtype=np.float64)[shard.local]
    E, gv, gR = backend.grad(shard.local_wl, res_local, kT, nel)
    return E, comm.allreduce(gv), comm.allreduce(gR)


class GpuBackend:
    """The CUDA library through ``api`` (device tensors)."""

    def __init__(self, ctx):
        import torch
        from . import api
        self.ctx, self.api, self.xp = ctx, api, torch

    def layout(self, wl):
        return self.api.dg_layout(wl.problem, wl.params)

    def ingredients(self, wl, res):
        return self.api.dg_ingredients(self.ctx, wl.problem, wl.params, res)

    def blocks(self, wl, kv, tr, pe, alpha):
        return self.api.dg_blocks(self.ctx, wl.problem, wl.params, kv, tr, pe, alpha)

    def grad(self, wl, res, kT, nel):
        return self.api.alb_grad(self.ctx, wl.problem, wl.params, res, kT, nel)
