"""The end-to-end path (DGDFT_HOST_BUFFERS) against the device path on a small slab with a V_eff correction."""
import numpy as np
import pytest

from gpu_util import gpu_context
from test_gpu_grad import _case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


def test_host_buffers_give_the_device_results(ctx):
    """The end-to-end path (DGDFT_HOST_BUFFERS: the library stages host inputs and outputs) computes the
    same eigenpairs, ALBs and DG blocks as the device path, V_eff correction included."""
    from paper_2003_00407_gb300 import api
    w = _case()
    p, q = w.problem, w.params
    kw = dict(precision=0, cheb_degree=12, tol=1e-10, max_iter=400, keep_eigvec=False)
    rd = api.alb_generate(ctx, p, q, **kw)
    bd = api.dg_assemble(ctx, p, q, rd, 20.0).cpu().numpy()
    rh = api.alb_generate(ctx, p, q, host_buffers=True, **kw)
    bh = api.dg_assemble_host(ctx, p, q, rh, 20.0).numpy()
    # FP64 path; compared basis-invariantly, since the order of the FP64 atomic sums in the Gram matrices
    # may differ between runs
    from helpers import subspace_sine
    assert np.abs(rh.eigval.numpy() - rd.eigval.cpu().numpy()).max() <= 1e-11
    Ah, _ = api.alb_views(p, q, rh)
    Ad, _ = api.alb_views(p, q, rd)
    dV = float(np.prod(p.dom_h[0]))
    for k in range(p.n_elem):
        assert subspace_sine(Ad[k].cpu().numpy(), Ah[k].numpy(), dV) <= 1e-8
        n = int(q.n_alb[k])
        ed = np.linalg.eigvalsh(0.5 * (bd[k, 0, :n, :n] + bd[k, 0, :n, :n].T))
        eh = np.linalg.eigvalsh(0.5 * (bh[k, 0, :n, :n] + bh[k, 0, :n, :n].T))
        assert np.abs(ed - eh).max() <= 1e-8
