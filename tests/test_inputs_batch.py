"""The batching workload's generator (rpd_inputs.batch_shapes): seeded, every
shape a valid input mesh of the expected genus, sphere centres spread to the
stated minimum spacing, all on one grid."""
import numpy as np

from rpd_inputs import batch_shapes


def test_batch_shapes_are_valid_and_seeded():
    ws = batch_shapes(6, seed=7, tmin=1000, tmax=8000, smin=32, smax=400)
    again = batch_shapes(6, seed=7, tmin=1000, tmax=8000, smin=32, smax=400)
    assert len(ws) == 6
    assert len({w.grid_bits for w in ws}) == 1
    for w, v in zip(ws, again):
        assert np.array_equal(w.tets, v.tets) and np.array_equal(w.centers, v.centers)
        info = w.info
        assert info["orient_min"] > 0 and info["manifold"] and info["components"] == 1 and info["shells"] == 1
        assert 1 <= w.ns <= 400 and w.ns <= max(32, w.nt // 8)
        kind = w.name.split("_")[1]
        if kind == "torus":
            assert info["chi"] == 0
        elif kind.startswith("slab"):
            assert info["chi"] == 1 - int(kind[4:])
        # no two centres closer than 3/4 of the lattice spacing (within rounding)
        c = w.centers
        d2 = ((c[:, None, :] - c[None, :, :]) ** 2).sum(-1) + np.eye(len(c)) * 1e9
        edge = np.linalg.norm(w.verts[w.tets[:, 0]] - w.verts[w.tets[:, 1]], axis=1)
        assert np.sqrt(d2.min()) > 0.3 * np.median(edge)
