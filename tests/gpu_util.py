"""Shared set-up of the GPU parity tests."""
import numpy as np
import pytest


def gpu_context():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00407_gb300 import build, api
    build.build()
    return api.Context(0)


def packed_blocks(prob, counts, rng, dtype=np.float64):
    """Random packed [count][N_k] blocks for every element."""
    parts = [rng.normal(size=(int(c), int(np.prod(prob.elem_Qn[k])))) for k, c in enumerate(counts)]
    return parts, np.concatenate([p.ravel() for p in parts]).astype(dtype)
