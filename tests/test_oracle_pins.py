"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: numbers the
paper prints (golden fixtures with citations), closed forms, invariants and
special cases.  The mutation tests plant a known mistake in the exact oracle
and show that a pin catches it.
"""
import json
import os
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

from oracle.tiny import rpd_exact, from_workload, mesh_euler, power_distance
from rpd_inputs import tiny, tiny_set, ring_spheres

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _eq7(mutate=None):
    g = _load("eq7_fractional_euler.json")
    pts = [tuple(p) for p in g["points"]]
    tri = [tuple(t) for t in g["triangles"]]
    return g, rpd_exact(pts, tri, [tuple(c) for c in g["centers"]], g["weights"], mutate=mutate)


# ------------------------------------------------------------ paper examples
def test_eq7_worked_example():
    """Sec. 4.1.2, Eq. 7: chi(A_x) = chi(B_x) = 1/2 with the printed V, E, F."""
    g, r = _eq7()
    x = g["cell"]
    for t, name in ((0, "A_x"), (1, "B_x")):
        exp = g["expected"][name]
        V, E, F = r["wcount"][(t, x)]
        assert (V, E, F) == (Fraction(exp["V"]), Fraction(exp["E"]), Fraction(exp["F"]))
        assert r["chi_piece"][(t, (x,))] == Fraction(exp["chi"])
    assert r["chi"][(x,)] == Fraction(g["expected"]["chi_x"])


def test_torus_nerve_example():
    """Sec. 3.3, torus with 1, 2, 3 spheres (figure 'topo_fix')."""
    g = _load("torus_nerve_example.json")["cases"]
    r1 = rpd_exact(*from_workload(tiny("ring", 1, 0, spheres=ring_spheres(1))))
    assert r1["chi"][(0,)] == g["1"]["rpc"]["chi"] and r1["beta0"][(0,)] == g["1"]["rpc"]["beta0"]
    r2 = rpd_exact(*from_workload(tiny("ring", 2, 0, spheres=ring_spheres(2))))
    for i in (0, 1):
        assert r2["chi"][(i,)] == g["2"]["rpc"]["chi"] and r2["beta0"][(i,)] == g["2"]["rpc"]["beta0"]
    assert r2["beta0"][(0, 1)] == g["2"]["rpf_beta0"]
    assert not r2["flag"][(0, 1)]
    r3 = rpd_exact(*from_workload(tiny("ring", 3, 0, spheres=ring_spheres(3))))
    assert all(r3["flag"].values()) == g["3"]["all_contractible"]
    assert sum(1 for k in r3["chi"] if len(k) == 3) == g["3"]["n_rpe"]


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("shape", ["box", "block", "ring"])
def test_single_sphere_gives_mesh_euler(shape):
    """One sphere: RPC = the whole shape, so chi(RPC) = V - E + F - T of the mesh."""
    w = tiny(shape, 1, 3)
    r = rpd_exact(*from_workload(w))
    assert r["chi"][(0,)] == mesh_euler([tuple(t) for t in w.tets]) == w.info["chi"]
    assert r["beta0"][(0,)] == 1


def _cases():
    return tiny_set(9)


@pytest.fixture(scope="module")
def exact_results():
    return [(w, rpd_exact(*from_workload(w))) for w in _cases()]


def test_pieces_partition_each_tet_exactly(exact_results):
    """Sum over spheres of vol P(t,i) = vol(t) and the same for first moments."""
    for w, r in exact_results:
        q, _, _ = w.ints()
        for t, simp in enumerate(w.tets):
            P = [tuple(int(v) for v in q[a]) for a in simp]
            rows = [[P[a][k] - P[0][k] for k in range(3)] for a in (1, 2, 3)]
            det = (rows[0][0] * (rows[1][1] * rows[2][2] - rows[1][2] * rows[2][1])
                   - rows[0][1] * (rows[1][0] * rows[2][2] - rows[1][2] * rows[2][0])
                   + rows[0][2] * (rows[1][0] * rows[2][1] - rows[1][1] * rows[2][0]))
            vol = Fraction(det, 6)
            mom = [vol * Fraction(sum(p[k] for p in P), 4) for k in range(3)]
            got = [v for (tt, i), v in r["pieces"].items() if tt == t]
            assert sum(v[0] for v in got) == vol
            for k in range(3):
                assert sum(v[1][k] for v in got) == mom[k]


def test_piece_centroid_belongs_to_its_cell(exact_results):
    """Brute force: the centroid of P(t,i) is strictly closer (in power
    distance) to sphere i than to every other sphere (Eq. 1)."""
    for w, r in exact_results:
        _, c, rad = w.ints()
        cw = [(tuple(int(v) for v in c[s]), int(rad[s]) ** 2) for s in range(w.ns)]
        for (t, i), (vol, mom) in r["pieces"].items():
            x = tuple(m / vol for m in mom)
            di = power_distance(x, *cw[i])
            assert all(di < power_distance(x, *cw[k]) for k in range(w.ns) if k != i)


def test_each_convex_piece_has_euler_one(exact_results):
    """Euler's polyhedron formula: V - E + F - C = 1 for every convex piece."""
    for _, r in exact_results:
        assert all(v == 1 for v in r["chi_plain"].values())


def test_inclusion_exclusion_gives_mesh_euler(exact_results):
    """Nerve / inclusion-exclusion (Sec. 3.3): sum chi(RPC) - sum chi(RPF)
    + sum chi(RPE) - #RPV = chi(shape)."""
    for w, r in exact_results:
        tot = sum((-1) ** (len(k) - 1) * v for k, v in r["chi"].items())
        assert tot == w.info["chi"]


def test_owner_rule_equals_fractional_rule(exact_results):
    for _, r in exact_results:
        for k, v in r["chi"].items():
            assert v.denominator == 1 and r["chi_own"][k] == v


def test_convex_domain_every_element_contractible():
    """A convex shape cut by power cells gives convex elements: all chi = 1 and
    beta0 = 1 (Sec. 3.3, contractibility test of Eq. 5-6)."""
    for seed in (11, 12):
        r = rpd_exact(*from_workload(tiny("box", 7, seed)))
        assert r["chi"] and all(r["flag"].values())


def test_torus_two_sphere_rpf_has_two_components():
    r = rpd_exact(*from_workload(tiny("ring", 2, 0, spheres=ring_spheres(2))))
    assert r["beta0"][(0, 1)] == 2 and r["chi"][(0, 1)] == 2


# ------------------------------------------------------- planted mistakes
def test_mutation_unit_weights_is_caught():
    g, r = _eq7(mutate="unit_weights")
    assert r["chi_piece"][(0, (g["cell"],))] != Fraction(g["expected"]["A_x"]["chi"])


def test_mutation_drop_cell_term_is_caught():
    w = tiny("box", 1, 3)
    r = rpd_exact(*from_workload(w), mutate="drop_cell")
    assert r["chi"][(0,)] != w.info["chi"]


def test_mutation_wrong_side_is_caught():
    w = tiny("box", 4, 21)
    r = rpd_exact(*from_workload(w), mutate="wrong_side")
    _, c, rad = w.ints()
    cw = [(tuple(int(v) for v in c[s]), int(rad[s]) ** 2) for s in range(w.ns)]
    bad = 0
    for (t, i), (vol, mom) in r["pieces"].items():
        x = tuple(m / vol for m in mom)
        di = power_distance(x, *cw[i])
        bad += not all(di < power_distance(x, *cw[k]) for k in range(w.ns) if k != i)
    assert bad > 0


def test_mutation_skip_last_sphere_is_caught():
    w = tiny("box", 5, 22)
    r = rpd_exact(*from_workload(w), mutate="skip_last")
    q, _, _ = w.ints()
    tot = sum(v[0] for v in r["pieces"].values())
    exact = Fraction(0)
    for simp in w.tets:
        P = [q[a].astype(object) for a in simp]
        m = np.array([P[1] - P[0], P[2] - P[0], P[3] - P[0]], dtype=object)
        exact += Fraction(int(m[0, 0] * (m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1])
                              - m[0, 1] * (m[1, 0] * m[2, 2] - m[1, 2] * m[2, 0])
                              + m[0, 2] * (m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0])), 6)
    assert tot != exact
