"""The synthetic input recipe: sizes, seeds and value ranges of the five configurations."""
import numpy as np

from workloads import make_config
from workloads.configs import n_blk_rule, probe_directions, probe_points


def test_sheet_recipe():
    w = make_config(5)
    p, q = w.problem, w.params
    assert p.n_elem == 1024 and p.n_atoms == 4096
    assert tuple(p.dom_n[0]) == (512, 512, 48) and np.allclose(p.dom_h, 0.4)
    assert np.all(p.elem_Qn == (32, 32, 48)) and np.all(p.elem_En == (16, 16, 48))
    assert np.all(q.n_eig == 72) and np.all(q.n_blk == 80) and np.all(q.n_alb == 64)
    assert p.n_stencil == 5 and p.n_proj_per_atom == 4 and p.r_cut == 3.2
    assert np.all((p.well_depth >= 2.0) & (p.well_depth <= 4.0)) and np.allclose(p.well_width, 0.8)
    assert np.all((p.proj_gamma >= 0.5) & (p.proj_gamma <= 2.0)) and np.allclose(p.proj_width, 0.8)
    assert np.allclose(w.n_electrons, 16.0)      # 4 atoms of 4 valence electrons per element
    # graphene-like areal density: 4 atoms per 6.4 x 6.4 bohr^2 = 0.35 atoms / A^2
    area_A2 = (16 * 0.4 * 0.529177) ** 2
    assert abs(4 / area_A2 - 0.35) < 0.02


def test_configs_are_seeded_and_reproducible():
    a, b = make_config(2), make_config(2)
    assert np.array_equal(a.problem.atom_pos, b.problem.atom_pos)
    assert np.array_equal(a.problem.proj_gamma, b.problem.proj_gamma)
    c = make_config(4)
    assert not np.array_equal(a.problem.atom_pos, c.problem.atom_pos)   # own seed


def test_uneven_batch_recipe():
    w = make_config(3)
    p, q = w.problem, w.params
    assert p.n_elem == 256 and p.n_stencil == 1
    shapes = {tuple(int(v) for v in s) for s in p.elem_Qn}
    assert all(s[0] in (24, 32, 40) and s[1] in (24, 32, 40) and s[2] in (32, 48) for s in shapes)
    assert len(shapes) == 18
    assert np.all((q.n_alb >= 20) & (q.n_alb <= 60))
    assert np.all(q.n_eig == np.ceil(1.25 * q.n_alb))
    assert np.all(q.n_blk == [n_blk_rule(int(n)) for n in q.n_eig])


def test_block_rule_and_probe_helpers():
    assert n_blk_rule(72) == 80 and n_blk_rule(40) == 48 and n_blk_rule(16) == 24
    d = probe_directions(3, 100, 1)
    assert d.shape == (3, 100) and np.allclose(np.linalg.norm(d, axis=1), 1.0)
    pts = probe_points(10, 50, 2)
    assert len(set(pts.tolist())) == 10 and pts.min() >= 0 and pts.max() < 50
