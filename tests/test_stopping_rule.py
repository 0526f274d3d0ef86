"""The per-pass stopping test of the CheFSI driver (Alg. CheFSI: iterate until the residuals of the
wanted Ritz pairs meet the tolerance), called through the library's exported host function
dgdft_stage_converged on synthetic residual histories.  No GPU is needed: the rule is plain host code
that the device bookkeeping kernel shares.

Rule under test (FP32 stage of the mixed path): leave at tol or tol_mixed; leave on stagnation (two
consecutive passes that each cut the residual by less than 20%) only at or below the FP32 rounding
floor 32 * 2^-24 * |b_up|; stagnation above that floor keeps the element iterating.
"""
import ctypes as C

import pytest

EPS32 = 2.0 ** -24
B_UP = 95.0                      # spectrum bound of a sheet element (Ha)
FLOOR = 32 * EPS32 * B_UP        # about 1.8e-4 Ha


@pytest.fixture(scope="module")
def lib():
    from paper_2003_00407_gb300 import build, _abi
    build.build()
    return _abi.load()


def run(lib, history, tol=1e-8, tol_mixed=1e-6, mixed=1, b_up=B_UP):
    """Feeds a residual history pass by pass; returns the 1-based pass that ends the stage (None = never)."""
    prev, stall = C.c_double(1e300), C.c_int(0)
    for i, r in enumerate(history):
        d = lib.dgdft_stage_converged(float(r), tol, tol_mixed, mixed, b_up, C.byref(prev), C.byref(stall))
        assert d in (0, 1)
        if d:
            return i + 1
    return None


def test_fp64_stage_stops_at_tol_only(lib):
    hist = [1e-1, 1e-3, 1e-5, 2e-8, 5e-9]
    assert run(lib, hist, tol=1e-8, mixed=0) == 5
    # stagnation never ends the FP64 stage
    assert run(lib, [1e-5] * 20, tol=1e-8, mixed=0) is None


def test_fp32_stage_stops_on_stagnation_at_the_floor(lib):
    # converging, then flat at the FP32 floor (about 3 eps |b_up|, as on the sheet elements)
    floor = 3 * EPS32 * B_UP
    hist = [1e-1, 1e-2, 1e-3, 1e-4, 1.2e-5] + [floor * (1 - 0.01 * i) for i in range(6)]
    # pass 6 is the first stagnating pass below the floor level, pass 7 the second
    assert run(lib, hist) == 7


def test_fp32_stage_keeps_going_when_stagnating_above_the_floor(lib):
    # a slowly converging element: 10% per pass from 1e-2, above the floor for the whole history
    hist = [1e-2 * 0.9 ** i for i in range(30)]
    assert min(hist) > FLOOR
    assert run(lib, hist) is None
    # stalls above the floor level do not count: an element that reaches the floor level still needs
    # two stagnating passes there
    hist2 = [2 * FLOOR * 0.9 ** i for i in range(6)] + [0.98 * FLOOR, 0.9 * FLOOR, 0.85 * FLOOR]
    assert run(lib, hist2) == 8


def test_fp32_stage_progress_resets_the_stall_count(lib):
    # stagnate once, improve by more than 20%, stagnate once: never two consecutive stalls
    f = 2 * EPS32 * B_UP
    hist = [1e-3, 10 * f, 9.5 * f, 5 * f, 4.9 * f, 2 * f, 1.95 * f, 1.0 * f, 0.99 * f]
    assert run(lib, hist) is None
    assert run(lib, hist + [0.98 * f]) == len(hist) + 1


def test_tolerances_and_non_finite_residuals_end_the_stage(lib):
    assert run(lib, [1e-3, 5e-7], tol_mixed=1e-6) == 2          # tol_mixed
    assert run(lib, [1e-3, 5e-9], tol_mixed=0.0) == 2           # tol
    assert run(lib, [1e-3, float("nan")]) == 2                   # NaN
    assert run(lib, [1e-3, float("inf")], mixed=0) == 2          # Inf


def test_floor_scales_with_the_spectrum_bound(lib):
    # the same stagnating history ends the stage for a wide spectrum but not for a narrow one
    hist = [1e-2, 1e-3, 3e-4, 3e-4, 3e-4]
    assert run(lib, hist, b_up=95.0) is None      # floor 1.8e-4: stagnation above it
    assert run(lib, hist, b_up=200.0) == 5        # floor 3.8e-4: the two stalls end the stage


def test_null_state_is_rejected(lib):
    prev = C.c_double(1.0)
    assert lib.dgdft_stage_converged(1.0, 0.0, 0.0, 1, 1.0, C.byref(prev), None) < 0
