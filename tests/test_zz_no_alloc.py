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


def _setup(torch):
    from paper_2003_00407_gb300 import api, _abi
    w = make_slab(3, 3, (16, 16, 48), (32, 32, 48), 0.4, 12, 8, 7)   # 9 elements, wells + projectors
    p, q = w.problem, w.params
    total = int(np.sum(q.n_blk.astype(np.int64) * np.prod(p.elem_Qn, axis=1)))
    v = api.v_extra_tensor(p, torch.device("cuda", 0))
    m = api.Marshalled(p, q, precision=_abi.MIXED, cheb_degree=10, tol=1e-8, max_iter=10, v_extra=v.data_ptr())
    return w, total, v, m


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import gpu_context
    from paper_2003_00407_gb300 import api, _abi
    ctx = gpu_context()
    lib = _lib()
    w, total, v, m = _setup(torch)
    p, q = w.problem, w.params
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(11)
    for call in range(2):
        X = torch.randn(total, dtype=torch.float32, device="cuda", generator=gen)
        ref = api.apply_hamiltonian(ctx, p, q, X, precision=_abi.MIXED)
        Y = torch.full_like(X, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        r = lib.dgdft_apply_hamiltonian_noalloc(C.byref(m.prob), C.byref(m.params), C.c_void_p(X.data_ptr()),
                                                C.c_void_p(Y.data_ptr()), stream)
        free1 = torch.cuda.mem_get_info()[0]
        assert r == 0, lib.dgdft_last_error(None)
        # the library's device array was set up by the first call (or by an earlier test); from then on
        # a call takes no device memory at all
        if call == 1:
            assert free1 == free0, (free0, free1)
        err = float((Y - ref).abs().max() / ref.abs().max())
        assert err <= FP32_TOL, (call, err)


_FRESH = r"""
import ctypes as C, sys
import numpy as np, torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from paper_2003_00407_gb300 import api, _abi
from test_zz_no_alloc import _setup, FP32_TOL
lib = _abi.load()
w, total, v, m = _setup(torch)
p, q = w.problem, w.params
X = torch.randn(total, dtype=torch.float32, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
Y = torch.full_like(X, float("nan"))
stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
# first call of the process: nothing of the library has run on this device yet
r = lib.dgdft_apply_hamiltonian_noalloc(C.byref(m.prob), C.byref(m.params), C.c_void_p(X.data_ptr()),
                                        C.c_void_p(Y.data_ptr()), stream)
assert r == 0, lib.dgdft_last_error(None)
ctx = api.Context(0)
ref = api.apply_hamiltonian(ctx, p, q, X, precision=_abi.MIXED)
err = float((Y - ref).abs().max() / ref.abs().max())
assert err <= FP32_TOL, err
print("fresh-process first call OK", err)
"""


@pytest.mark.gpu
def test_noalloc_as_first_call_of_a_fresh_process():
    """The allocation-free entry point does its own per-device set-up (device address of its array,
    twiddles, shared-memory limit) when it is the first call of a process, before any context."""
    import os
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib()
    here = os.path.dirname(os.path.abspath(__file__))
    code = _FRESH.format(root=os.path.dirname(here), tests=here)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "fresh-process first call OK" in out.stdout


@pytest.mark.gpu
def test_noalloc_reports_non_finite_v_extra():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00407_gb300 import _abi
    lib = _lib()
    w, total, v, m = _setup(torch)
    v[1234] = float("nan")          # a point inside Q of some element
    X = torch.ones(total, dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    r = lib.dgdft_apply_hamiltonian_noalloc(C.byref(m.prob), C.byref(m.params), C.c_void_p(X.data_ptr()),
                                            C.c_void_p(Y.data_ptr()),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert r == _abi.BAD_INPUT
    assert b"not finite" in lib.dgdft_last_error(None)
