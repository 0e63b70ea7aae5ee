"""The CPU thinning (oracle/thin.py, Sec. 5.3) and the oracle's RPE lengths,
pinned without the library: a hand-derived single-tetrahedron thinning
(tests/golden/thinning_single_tet.json), Euler-characteristic invariance of
simple-pair removal, and the length of a radical line crossing a box."""
import json
import os
from itertools import combinations

import numpy as np

import oracle
from oracle.thin import thin
from rpd_inputs import tiny

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    with open(os.path.join(HERE, "golden", "thinning_single_tet.json")) as f:
        return json.load(f)


def test_single_tet_by_hand():
    g = _load()
    faces = [tuple(f) for f in g["faces"]]
    alpha = dict(zip(faces, g["alpha"]))
    e, f, t = thin(g["edges"], g["faces"], alpha, g["tets"], g["sigma"])
    assert [list(x) for x in e] == g["expected_edges"]
    assert [list(x) for x in f] == g["expected_faces"] and t == []
    e, f, t = thin(g["edges"], g["faces"], alpha, g["tets"], 0.25)
    assert [list(x) for x in f] == g["sigma_0_25_expected_faces"]
    assert [list(x) for x in e] == g["sigma_0_25_expected_edges"]


def test_thinning_keeps_euler_characteristic():
    rng = np.random.default_rng(4)
    for _ in range(20):
        # a random pure complex: a few tets on 7 vertices and their closure
        tets = sorted({tuple(sorted(rng.choice(7, 4, replace=False).tolist())) for _ in range(5)})
        faces = sorted({f for t in tets for f in combinations(t, 3)} |
                       {tuple(sorted(rng.choice(7, 3, replace=False).tolist())) for _ in range(3)})
        edges = sorted({e for f in faces for e in combinations(f, 2)})
        verts = sorted({v for e in edges for v in e})
        alpha = {f: float(rng.uniform()) for f in faces}
        e2, f2, t2 = thin(edges, faces, alpha, tets, 0.7)
        chi0 = len(verts) - len(edges) + len(faces) - len(tets)
        assert len(verts) - len(e2) + len(f2) - len(t2) == chi0


def test_radical_line_length_across_a_box():
    """Three equal spheres with centres on a horizontal circle: their radical
    line is the vertical line through the circle's centre, so in the 2x2x2
    box the one restricted power edge has length 2 (box height)."""
    th = 2 * np.pi * np.arange(3) / 3 + 0.3
    c = np.stack([1.0137 + 0.6 * np.cos(th), 0.9781 + 0.6 * np.sin(th), np.full(3, 1.0)], axis=1)
    w = tiny("box", 3, 0, spheres=(c, np.full(3, 0.5)))
    o = oracle.run(w)
    e = o["kinds"][3]
    assert e["keys"].tolist() == [[0, 1, 2]]
    assert abs(e["length"][0] / float(1 << w.grid_bits) - 2.0) < 1e-9
