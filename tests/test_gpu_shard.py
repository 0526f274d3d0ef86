"""Element sharding on the GPU (Sec. II.B), two ranks emulated phase by phase in one process on one GPU.

Each emulated rank generates the ALBs of its own elements, forms their DG ingredients through the C-ABI
(dgdft_dg_ingredients), packs the face and overlap records its neighbour rank needs, and -- after the
records are handed over in memory, which stands in for the point-to-point exchange -- forms the blocks of
its elements with dgdft_dg_blocks.  No kernel of one rank waits on another: the ranks run one after the
other.  The blocks equal those of one dgdft_dg_assemble call over all elements, and the per-rank
gradients summed over ranks equal one dgdft_alb_grad call.
"""
import numpy as np
import pytest
import torch

from gpu_util import gpu_context
from workloads.configs import make_slab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


def _slab():
    w = make_slab(4, 2, (8, 6, 12), (16, 12, 12), 0.45, 10, 6, 5, r_cut=2.6, width=0.7, proj_width=0.7)
    w.alpha = 20.0
    return w


@pytest.mark.parametrize("precision", [0, 1])
def test_two_emulated_ranks_match_one_call(ctx, precision):
    from paper_2003_00407_gb300 import api, shard
    w = _slab()
    kw = dict(precision=precision, cheb_degree=12, tol=1e-9, max_iter=300)
    # single call over all elements
    res = api.alb_generate(ctx, w.problem, w.params, **kw)
    ref = api.dg_assemble(ctx, w.problem, w.params, res, w.alpha).cpu().numpy()
    nel = np.full(w.problem.n_elem, 4.0)
    E_ref, gv_ref, gR_ref = (t.cpu().numpy() for t in api.alb_grad(ctx, w.problem, w.params, res, 0.01, nel))
    world = 2
    be = shard.GpuBackend(ctx)
    shards = [shard.Shard(w, world, r) for r in range(world)]
    results, states = [], []
    for sh in shards:                                   # phase 1: generation, ingredients, sends
        # each rank's generation covers its own elements only; its random start is numbered by the
        # element's place in the call, so a separate call converges to the same ALBs only within the
        # solver tolerance -- the blocks are compared bit-near-exactly on the one-call ALBs instead
        own = api.alb_generate(ctx, sh.local_wl.problem, sh.local_wl.params, **kw)
        assert int(own.status.abs().sum()) == 0
        r_loc = api.result_subset(res, w.problem, w.params, sh.local, sh.local_wl.problem, sh.local_wl.params,
                                  precision=precision)
        results.append(r_loc)
        states.append(shard.dg_prepare(sh, be, r_loc))
    mail = {(r, q): states[r]["sends"][q] for r in range(world) for q in shards[r].peers}
    gsum_v, gsum_R = 0.0, 0.0
    for r, sh in enumerate(shards):                     # phase 2: receive, blocks, gradient parts
        recvs = {q: mail[(q, r)] for q in sh.peers}
        for q in sh.peers:
            assert recvs[q].numel() == states[r]["sizes"][q]
        blocks = shard.dg_finish(sh, be, states[r], recvs).cpu().numpy()
        L = ref.shape[2]
        err = np.abs(blocks[:, :, :L, :L] - ref[sh.local]).max()
        assert err <= 1e-10 * np.abs(ref).max(), (r, err)
        E, gv, gR = api.alb_grad(ctx, sh.local_wl.problem, sh.local_wl.params, results[r], 0.01, nel[sh.local])
        assert np.abs(E.cpu().numpy() - E_ref[sh.local]).max() <= 1e-10
        gsum_v = gsum_v + gv.cpu().numpy()
        gsum_R = gsum_R + gR.cpu().numpy()
    assert np.abs(gsum_v - gv_ref).max() <= 1e-10 * np.abs(gv_ref).max()
    assert np.abs(gsum_R - gR_ref).max() <= 1e-10 * np.abs(gR_ref).max()


def test_ingredients_then_blocks_equal_assemble(ctx):
    """dgdft_dg_ingredients + dgdft_dg_blocks in a row give the blocks of dgdft_dg_assemble, bit for bit."""
    from paper_2003_00407_gb300 import api
    w = _slab()
    res = api.alb_generate(ctx, w.problem, w.params, precision=0, cheb_degree=12, tol=1e-9, max_iter=300)
    ref = api.dg_assemble(ctx, w.problem, w.params, res, w.alpha)
    kv, tr, pe = api.dg_ingredients(ctx, w.problem, w.params, res)
    got = api.dg_blocks(ctx, w.problem, w.params, kv, tr, pe, w.alpha)
    assert torch.equal(got, ref)
