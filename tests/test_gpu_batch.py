"""Batched builds (rpd_build_batch) through the C-ABI: every shape's rows of
every table, and its pieces, must equal those of rpd_build on that shape
alone, with the ids shifted by the shape's offsets; bad batches must be
rejected."""
import numpy as np
import pytest
import torch

from paper_2403_18761_gb300 import rpd_build, rpd_build_batch, RpdError
from paper_2403_18761_gb300.rpd import collect, RPD_E_INVALID
from rpd_inputs import torus_c1, block_c2, genus_slab, tiny, ring_spheres

pytestmark = pytest.mark.gpu

G = 18   # one grid for the whole batch


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _shapes():
    ws = [torus_c1(), genus_slab(2, h=0.15, ns=64), tiny("ring", 3, 0, spheres=ring_spheres(3)),
          block_c2(h=0.15, ns=300), genus_slab(5, h=0.15, ns=200), tiny("box", 7, 5)]
    return [(w.verts, w.tets, w.centers, w.radii) for w in ws]


def _single(shape, precision, k):
    v, t, c, r = shape
    return collect(rpd_build(v, t, c, r, precision=precision, k=k, grid_bits=G))


@pytest.mark.parametrize("precision,k", [("fp32", 32), ("fp64", 16)])
def test_batch_equals_single_builds(precision, k):
    shapes = _shapes()
    ctx = rpd_build_batch(shapes, precision=precision, k=k, grid_bits=G)
    got = collect(ctx)
    soff, toff = ctx.batch["sphere_off"], ctx.batch["tet_off"]
    offs = {kind: ctx.shape_offsets(kind) for kind in (0, 1, 2, 3, 4)}
    for s, shape in enumerate(shapes):
        want = _single(shape, precision, k)
        for kind in (1, 2, 3, 4):
            a, b = offs[kind][s], offs[kind][s + 1]
            g = got["kinds"][kind]
            w = want["kinds"][kind]
            assert np.array_equal(g["keys"][a:b] - soff[s], w["keys"]), (s, kind)
            for f in ("chi", "beta0", "flag"):
                assert np.array_equal(g[f][a:b], w[f]), (s, kind, f)
        a, b = offs[0][s], offs[0][s + 1]
        assert np.array_equal(got["tet"][a:b] - toff[s], want["tet"]), s
        assert np.array_equal(got["sphere"][a:b] - soff[s], want["sphere"]), s
        assert np.array_equal(got["vol"][a:b], want["vol"]), s
        assert np.array_equal(got["moment"][a:b], want["moment"]), s
    for kind in (0, 1, 2, 3, 4):
        assert offs[kind][-1] == (len(got["tet"]) if kind == 0 else len(got["kinds"][kind]["keys"]))


def test_batch_of_one_is_a_build():
    shapes = _shapes()[:1]
    got = collect(rpd_build_batch(shapes, grid_bits=G, k=32))
    want = _single(shapes[0], "fp32", 32)
    for kind in (1, 2, 3, 4):
        assert np.array_equal(got["kinds"][kind]["keys"], want["kinds"][kind]["keys"])
    assert np.array_equal(got["vol"], want["vol"])


def test_batch_rejects_cross_shape_tets_and_bad_offsets():
    shapes = _shapes()[:2]
    v, t, c, r = shapes[1]
    bad = (v, np.asarray(t) - 3, c, r)   # reaches into the previous shape's vertices
    with pytest.raises(RpdError) as e:
        rpd_build_batch([shapes[0], bad], grid_bits=G)
    assert e.value.status == RPD_E_INVALID
    with pytest.raises(RpdError) as e:   # a shape without spheres
        rpd_build_batch([shapes[0], (v, t, c[:0], r[:0])], grid_bits=G)
    assert e.value.status == RPD_E_INVALID
    # the context still works after rejected batches
    ok = collect(rpd_build_batch(shapes, grid_bits=G))
    assert len(ok["tet"]) > 0


def test_autotuner_picks_a_k_that_gives_the_same_diagram():
    from paper_2403_18761_gb300 import rpd_autotune
    w = block_c2(h=0.15, ns=300)
    k, ms = rpd_autotune(w.verts, w.tets, w.centers, w.radii, ks=(4, 8, 16, 32), reps=2, grid_bits=w.grid_bits)
    assert k in (4, 8, 16, 32) and ms > 0
    a = collect(rpd_build(w.verts, w.tets, w.centers, w.radii, k=k, grid_bits=w.grid_bits))
    b = collect(rpd_build(w.verts, w.tets, w.centers, w.radii, k=32, grid_bits=w.grid_bits))
    for kind in (1, 2, 3, 4):
        for f in ("keys", "chi", "beta0", "flag"):
            assert np.array_equal(a["kinds"][kind][f], b["kinds"][kind][f])
    assert np.array_equal(a["vol"], b["vol"])
