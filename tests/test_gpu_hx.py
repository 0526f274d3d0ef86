"""GPU parity of the hot operator H x (Eq. LocalKS) and the Chebyshev filter (Alg. CheFSI step 2)."""
import numpy as np
import pytest
import torch

from oracle import local_operator as lo, chefsi as cf
from workloads import make_config
from workloads.configs import make_slab, make_cube
from gpu_util import gpu_context, packed_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


CASES = {
    "cube16_wells": lambda: make_config(1),
    "slab_proj_small": lambda: make_slab(3, 2, (8, 6, 12), (16, 12, 12), 0.45, 6, 4, 5, r_cut=2.6,
                                         width=0.7, proj_width=0.7),
    "slab_q32x32x48": lambda: make_slab(3, 3, (16, 16, 48), (32, 32, 48), 0.4, 12, 8, 7),
    # Q shapes whose FP32 step runs on a CTA pair (half spectrum over two CTAs); Q = the whole periodic
    # box in x and y, so projector boxes wrap around
    "slab_q40x40x48_pair": lambda: make_slab(2, 2, (20, 20, 48), (40, 40, 48), 0.4, 12, 8, 9),
    "slab_q40x32x48_pair": lambda: make_slab(2, 2, (20, 16, 48), (40, 32, 48), 0.4, 12, 8, 11),
    "cube_odd_radix": lambda: make_cube(3, n=20, L=9.0, n_wells=4, n_proj=4, En=10, n_eig=6, n_alb=4),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_apply_hamiltonian_matches_oracle(ctx, case, precision):
    from paper_2003_00407_gb300 import api
    w = CASES[case]()
    p, q = w.problem, w.params
    rng = np.random.default_rng(0)
    parts, flat = packed_blocks(p, q.n_blk, rng, np.float64 if precision == 0 else np.float32)
    X = torch.as_tensor(flat, device="cuda")
    Y = api.apply_hamiltonian(ctx, p, q, X, precision=precision).cpu().numpy().astype(np.float64)
    o = 0
    tol = 1e-12 if precision == 0 else 3e-6
    for k in range(p.n_elem):
        op = lo.LocalOperator(p, k)
        ref = op.apply(parts[k].astype(np.float32).astype(np.float64) if precision else parts[k])
        got = Y[o:o + ref.size].reshape(ref.shape)
        o += ref.size
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < tol, (case, k, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_chebyshev_filter_matches_oracle(ctx, precision):
    from paper_2003_00407_gb300 import api
    w = CASES["slab_proj_small"]()
    p, q = w.problem, w.params
    rng = np.random.default_rng(1)
    parts, flat = packed_blocks(p, q.n_blk, rng, np.float64 if precision == 0 else np.float32)
    bounds = np.array([[-1.0 - 0.1 * k, 2.0 + 0.05 * k, 60.0 + k] for k in range(p.n_elem)])
    m = 7
    Y = api.chebyshev_filter(ctx, p, q, torch.as_tensor(flat, device="cuda"), bounds, m,
                             precision=precision).cpu().numpy().astype(np.float64)
    o = 0
    for k in range(p.n_elem):
        op = lo.LocalOperator(p, k)
        X = parts[k].astype(np.float32).astype(np.float64) if precision else parts[k]
        ref = cf.chebyshev_filter(op, X, m, bounds[k, 1], bounds[k, 2], bounds[k, 0])
        got = Y[o:o + ref.size].reshape(ref.shape)
        o += ref.size
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < (1e-11 if precision == 0 else 2e-5), (k, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_hamiltonian_reports_non_finite_v_extra(ctx, precision):
    from paper_2003_00407_gb300 import api
    w = CASES["slab_proj_small"]()
    p, q = w.problem, w.params
    p.v_extra = p.v_extra.copy()
    p.v_extra[7] = np.nan
    rng = np.random.default_rng(2)
    _, flat = packed_blocks(p, q.n_blk, rng, np.float64 if precision == 0 else np.float32)
    with pytest.raises(api.DgdftError) as e:
        api.apply_hamiltonian(ctx, p, q, torch.as_tensor(flat, device="cuda"), precision=precision)
    assert "BAD_INPUT" in str(e.value) and "not finite" in str(e.value)
