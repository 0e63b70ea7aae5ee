"""Seeded generators: meshes satisfy the paper's input assumption (Sec. 3.3)."""
import numpy as np
import pytest

from rpd_inputs import torus_c1, tiny, tiny_set, validate, snap


def test_torus_c1_mesh_is_a_solid_torus():
    w = torus_c1()
    info = w.info
    assert 4000 < w.nt < 6500
    assert w.ns == 64
    assert info["orient_min"] == 1 and info["manifold"] and info["components"] == 1 and info["shells"] == 1
    assert info["chi"] == 0


def test_torus_c1_is_deterministic():
    a, b = torus_c1(), torus_c1()
    assert np.array_equal(a.tets, b.tets) and np.array_equal(a.verts, b.verts)
    assert np.array_equal(a.centers, b.centers) and np.array_equal(a.radii, b.radii)


def test_inputs_lie_on_the_grid():
    w = torus_c1()
    s = float(1 << w.grid_bits)
    for arr in (w.verts, w.centers, w.radii):
        assert np.all(arr * s == np.rint(arr * s))
    q, c, r = w.ints()
    assert np.abs(q).max() < (1 << 21) and np.abs(c).max() < (1 << 21)


@pytest.mark.parametrize("shape,chi", [("box", 1), ("block", 1), ("ring", 0)])
def test_tiny_shapes(shape, chi):
    w = tiny(shape, 3, 7)
    assert w.info["chi"] == chi and w.info["manifold"] and w.info["shells"] == 1


def test_tiny_set_sizes():
    ws = tiny_set(12)
    assert all(w.nt <= 48 and 1 <= w.ns <= 12 for w in ws)
