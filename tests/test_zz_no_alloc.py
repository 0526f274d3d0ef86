"""The allocation-free H x entry point (dgdft_apply_hamiltonian_noalloc).

Some callers cannot allocate device memory (their HBM is reserved by another
allocator, or they cannot accept cudaMalloc's device-wide synchronisation).
This entry point serves them from a fixed scratch array inside the library; its
output must match the allocating dgdft_apply_hamiltonian within the FP32
tolerance of the other H x tests, on consecutive calls that reuse the array.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import make_config
from workloads.configs import make_slab

FP32_TOL = 3e-6   # relative, as in tests/test_gpu_hx.py


def _lib():
    from paper_2003_00407_gb300 import build, _abi
    build.build()
    return _abi.load()


def test_oversized_problem_is_rejected_before_any_gpu_work():
    from paper_2003_00407_gb300 import api, _abi
    lib = _lib()
    w = make_config(5)   # 1024 elements: far beyond the fixed scratch
    m = api.Marshalled(w.problem, w.params, precision=_abi.MIXED, cheb_degree=80, tol=1e-8, max_iter=10)
    dummy = C.c_void_p(16)   # never dereferenced: the size check comes first
    r = lib.dgdft_apply_hamiltonian_noalloc(C.byref(m.prob), C.byref(m.params), dummy, dummy, None)
    assert r == _abi.UNSUPPORTED
    assert b"bytes of scratch" in lib.dgdft_last_error(None)


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import gpu_context
    from paper_2003_00407_gb300 import api, _abi
    ctx = gpu_context()
    lib = _lib()
    w = make_slab(3, 3, (16, 16, 48), (32, 32, 48), 0.4, 12, 8, 7)   # 9 elements, wells + projectors
    p, q = w.problem, w.params
    total = int(np.sum(q.n_blk.astype(np.int64) * np.prod(p.elem_Qn, axis=1)))
    v = api.v_extra_tensor(p, torch.device("cuda", 0))
    m = api.Marshalled(p, q, precision=_abi.MIXED, cheb_degree=10, tol=1e-8, max_iter=10, v_extra=v.data_ptr())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(11)
    for call in range(2):
        X = torch.randn(total, dtype=torch.float32, device="cuda", generator=gen)
        ref = api.apply_hamiltonian(ctx, p, q, X, precision=_abi.MIXED)
        Y = torch.full_like(X, float("nan"))
        r = lib.dgdft_apply_hamiltonian_noalloc(C.byref(m.prob), C.byref(m.params), C.c_void_p(X.data_ptr()),
                                                C.c_void_p(Y.data_ptr()), stream)
        assert r == 0, lib.dgdft_last_error(None)
        err = float((Y - ref).abs().max() / ref.abs().max())
        assert err <= FP32_TOL, (call, err)
