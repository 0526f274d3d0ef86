"""Gram matrices of FP32 blocks on the tcgen05 tensor cores (3xTF32; the overlap and projection matrices
of the Cholesky-QR and Rayleigh-Ritz steps of Alg. CheFSI in the FP32 stage) against the exact FP64
products of the same FP32 inputs.  Bound: 2^-18 of dV sum_p |x_ip| |y_jp| per entry (the split leaves a
few 2^-22 per product; the tensor cores accumulate 64 points in FP32 before the exact two-sum)."""
import numpy as np
import pytest
import torch

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return gpu_context()


def packed(rng, rows, pts, scale=1.0):
    blocks = [(rng.standard_normal((r, p)) * scale).astype(np.float32) for r, p in zip(rows, pts)]
    off = np.cumsum([0] + [b.size for b in blocks])[:-1]
    return blocks, off, torch.as_tensor(np.concatenate([b.ravel() for b in blocks]), device="cuda")


def check(G, bx, by, dV, ldg):
    for k in range(len(bx)):
        x, y = bx[k].astype(np.float64), by[k].astype(np.float64)
        ref = dV[k] * (x @ y.T)
        bound = dV[k] * (np.abs(x) @ np.abs(y).T) * 2.0 ** -18
        got = G[k, :x.shape[0], :y.shape[0]]
        assert np.all(np.abs(got - ref) <= bound + 1e-300), (k, np.abs(got - ref).max(), bound.min())
        rest = G[k].copy()
        rest[:x.shape[0], :y.shape[0]] = 0.0
        assert np.all(rest == 0.0)


@pytest.mark.parametrize("rows,pts", [
    ([80, 80], [49152, 49152]),          # sheet element blocks (12 chunks of 4096 points)
    ([12, 7, 96, 1], [1000, 4099, 5003, 33]),   # ragged: tails inside a stage, chunk and period
    ([16, 48], [8000, 6144]),
])
def test_gram_xx(ctx, rows, pts):
    from paper_2003_00407_gb300 import api
    rng = np.random.default_rng(len(rows) * 7 + rows[0])
    bx, off, X = packed(rng, rows, pts)
    dV = rng.uniform(0.01, 0.1, len(rows))
    G = api.gram_fp32(ctx, X, off, rows, pts, dV, ldg=96).cpu().numpy()
    check(G, bx, bx, dV, 96)


def test_gram_xy_unaligned(ctx):
    """Different X and Y, element offsets that are not multiples of 4 floats (scalar load path)."""
    from paper_2003_00407_gb300 import api
    rng = np.random.default_rng(11)
    rows_x, rows_y, pts = [80, 33], [80, 65], [6001, 4097]
    bx = [rng.standard_normal((r, p)).astype(np.float32) for r, p in zip(rows_x, pts)]
    by = [(rng.standard_normal((r, p)) * 3.0).astype(np.float32) for r, p in zip(rows_y, pts)]
    xo = np.array([1, 1 + bx[0].size + 2])
    yo = np.array([3, 3 + by[0].size + 5])
    X = torch.zeros(int(xo[-1] + bx[1].size + 1), dtype=torch.float32)
    Y = torch.zeros(int(yo[-1] + by[1].size + 1), dtype=torch.float32)
    for k in range(2):
        X[xo[k]:xo[k] + bx[k].size] = torch.as_tensor(bx[k].ravel())
        Y[yo[k]:yo[k] + by[k].size] = torch.as_tensor(by[k].ravel())
    dV = np.array([0.5, 0.25])
    G = api.gram_fp32(ctx, X.cuda(), xo, rows_x, pts, dV, Y=Y.cuda(), y_off=yo, ny=rows_y, ldg=80).cpu().numpy()
    check(G, bx, by, dV, 80)


def test_gram_precision_beyond_tf32(ctx):
    """Entries that a single TF32 product would get wrong at 1e-4: X with mantissas beyond 10 bits."""
    from paper_2003_00407_gb300 import api
    rng = np.random.default_rng(5)
    x = (1.0 + rng.uniform(0, 2.0 ** -12, (8, 4096))).astype(np.float32)
    G = api.gram_fp32(ctx, torch.as_tensor(x.ravel(), device="cuda"), [0], [8], [4096], [1.0]).cpu().numpy()[0]
    ref = x.astype(np.float64) @ x.astype(np.float64).T
    assert np.abs(G - ref).max() / ref.max() < 4e-6


def test_gram_rejects_bad_rows(ctx):
    from paper_2003_00407_gb300 import api
    X = torch.zeros(200 * 10, dtype=torch.float32, device="cuda")
    with pytest.raises(api.DgdftError):
        api.gram_fp32(ctx, X, [0], [200], [10], [1.0])


@pytest.mark.parametrize("nin,nout,pts", [
    ([80, 80], [80, 80], [49152, 1000]),     # sheet blocks; a tail inside the last 128-point tile
    ([96, 7, 33], [96, 12, 1], [3000, 129, 1025]),   # K = 96 (one operand buffer), ragged counts
])
def test_rotate(ctx, nin, nout, pts):
    """Z_k = W_k^T X_k (X <- X W of Cholesky-QR and Rayleigh-Ritz) against FP64 products of the same inputs;
    bound 2^-18 of sum_i |W_ij| |X_ip|."""
    from paper_2003_00407_gb300 import api
    rng = np.random.default_rng(sum(nin) + len(pts))
    bx, off, X = packed(rng, nin, pts)
    ldw = 96
    W = np.zeros((len(nin), ldw, ldw))
    for k in range(len(nin)):
        W[k, :nin[k], :nout[k]] = rng.standard_normal((nin[k], nout[k]))
    Z, zo = api.rotate_fp32(ctx, X, off, nin, pts, torch.as_tensor(W, device="cuda"), nout)
    Z = Z.cpu().numpy()
    for k in range(len(nin)):
        w = W[k, :nin[k], :nout[k]]
        x = bx[k].astype(np.float64)
        ref = w.T @ x
        bound = (np.abs(w).T @ np.abs(x)) * 2.0 ** -18
        got = Z[zo[k]:zo[k] + nout[k] * pts[k]].reshape(nout[k], pts[k])
        assert np.all(np.abs(got - ref) <= bound + 1e-30), (k, np.abs(got - ref).max())


def test_rotate_in_place(ctx):
    """Z aliasing X (the Cholesky-QR use): every tile of X is read before its points are overwritten."""
    from paper_2003_00407_gb300 import api
    rng = np.random.default_rng(3)
    nin, pts = [64, 64], [4096 + 77, 2048]
    bx, off, X = packed(rng, nin, pts)
    W = torch.as_tensor(np.linalg.qr(rng.standard_normal((2, 64, 64)))[0], device="cuda")
    ref = [W[k].cpu().numpy().T @ bx[k].astype(np.float64) for k in range(2)]
    api.rotate_fp32(ctx, X, off, nin, pts, W, nin, Z=X, z_off=off)
    Xn = X.cpu().numpy()
    for k in range(2):
        got = Xn[off[k]:off[k] + bx[k].size].reshape(bx[k].shape)
        assert np.abs(got - ref[k]).max() < 1e-5 * np.abs(ref[k]).max()
