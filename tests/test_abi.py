"""The C-ABI library builds, loads and exports every entry point of include/dgdft.h (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_00407_gb300 import build, _abi
    build.build()
    return _abi.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dgdft.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(dgdft_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dgdft_alb_generate", "dgdft_dg_assemble", "dgdft_alb_grad", "dgdft_ctx_create",
              "dgdft_ctx_destroy", "dgdft_last_error", "dgdft_alb_query_sizes"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_query_sizes_on_host(lib):
    from workloads import make_config
    from paper_2003_00407_gb300 import api
    w = make_config(2)
    m = api.Marshalled(w.problem, w.params, precision=0, cheb_degree=40, tol=1e-8, max_iter=50)
    L, nalb, nvec, ncoef, ngrid, nblocks = api.query_sizes(m)
    assert L == 48
    assert nalb == 64 * 32 * 16 * 16 * 48
    assert nvec == 64 * 40 * 32 * 32 * 48
    assert ngrid == 128 * 128 * 48
    assert nblocks == 5 * 64 * 48 * 48


@pytest.mark.parametrize("mutate,code", [
    (lambda p, q: setattr(q, "n_alb", q.n_eig + 1), 1),           # n_alb > n_eig
    (lambda p, q: p.elem_Qn.__setitem__((0, 0), 33), 1),         # Qn - En odd
    (lambda p, q: p.elem_Qn.__setitem__(slice(None), (26, 32, 48)) or p.elem_En.__setitem__(slice(None), (16, 16, 48)), 8),  # 26 = 2*13
    (lambda p, q: setattr(p, "r_cut", 30.0), 1),                 # domain side < 2 r_cut
    (lambda p, q: q.n_blk.__setitem__(slice(None), q.n_eig - 1), 1),   # filter block smaller than n_eig
    (lambda p, q: q.n_blk.__setitem__(slice(None), 104) or q.n_eig.__setitem__(slice(None), 100), 8),  # block > 96
    (lambda p, q: p.dom_h.__setitem__((0, 0), 0.0), 1),          # zero grid spacing
    (lambda p, q: p.neighbors.__setitem__((0, 1), 9999), 1),     # neighbour id out of range
])
def test_query_sizes_rejects_bad_arguments(lib, mutate, code):
    import copy
    from workloads import make_config
    from paper_2003_00407_gb300 import api
    w = make_config(2)
    p, q = copy.deepcopy(w.problem), copy.deepcopy(w.params)
    mutate(p, q)
    m = api.Marshalled(p, q, precision=0, cheb_degree=40, tol=1e-8, max_iter=50)
    with pytest.raises(api.DgdftError) as e:
        api.query_sizes(m)
    assert e.value.code == code
    assert len(str(e.value)) > len("INVALID_ARG: dgdft_alb_query_sizes: ")   # the reason is reported


def test_query_sizes_rejects_an_empty_partition(lib):
    from workloads import make_config
    from workloads.configs import subset
    from paper_2003_00407_gb300 import api
    w = subset(make_config(2), [])
    w.problem.n_stencil = 1
    w.problem.neighbors = np.zeros((0, 1), dtype=np.int32)
    m = api.Marshalled(w.problem, w.params, precision=0, cheb_degree=40, tol=1e-8, max_iter=50)
    with pytest.raises(api.DgdftError) as e:
        api.query_sizes(m)
    assert e.value.code == 1


def test_context_creation_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.dgdft_ctx_create(C.byref(h), 0) == 7
    assert b"no CUDA device" in lib.dgdft_last_error(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the three C structs have the header's sizes and field offsets (compiled
    with the host C compiler)."""
    import shutil
    import subprocess
    from paper_2003_00407_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"dgdft_problem": _abi.Problem, "dgdft_alb_params": _abi.AlbParams, "dgdft_alb_result": _abi.AlbResult,
               "dgdft_dg_solve_params": _abi.DGSolveParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dgdft.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
