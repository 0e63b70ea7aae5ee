"""Partial RPD update, pin points, sphere shrinking and the topology-repair
loop on the GPU, through the C-ABI (Sec. 4 intro, 4.1.1, 4.1.2, 5.1, 5.2).

* rpd_insert must give exactly what rpd_build gives on the enlarged sphere
  set: every table, every piece, every volume bit for bit.
* rpd_shrink must match the CPU restatement (oracle/shrink.py) to 1e-9 of
  the radius.
* rpd_pins must pick the boundary triangles the paper's rules name.
* rpd_repair must end with every RPC, RPF and RPE contractible, as judged by
  the oracle run on the final sphere set.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.shrink import shrink as cpu_shrink, boundary_triangles
from oracle.tiny import rpd_exact, from_workload
from paper_2403_18761_gb300 import rpd_build, build_workload, RpdError
from paper_2403_18761_gb300.rpd import collect, RPD_E_INVALID
from rpd_inputs import torus_c1, block_c2, tiny, ring_spheres, genus_slab
from rpd_inputs.configs import Workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    oracle.build()


def _same(a, b, tag=""):
    for kind in (1, 2, 3, 4):
        for f in ("keys", "chi", "beta0", "flag"):
            assert np.array_equal(a["kinds"][kind][f], b["kinds"][kind][f]), (tag, kind, f)
    for f in ("tet", "sphere", "vol", "moment"):
        assert np.array_equal(a[f], b[f]), (tag, f)


def _sub(w, idx):
    return Workload(w.name, w.verts, w.tets, w.centers[idx], w.radii[idx], w.grid_bits, w.k, w.precision, w.info)


# --------------------------------------------------------- partial update
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_insert_one_at_a_time_equals_fresh_build(precision):
    w = torus_c1()
    base = 58
    ctx = build_workload(_sub(w, np.arange(base)), precision=precision)
    for n in range(base, w.ns):   # the last two cross 2^6 - 1 spheres: keys repacked
        ctx.rpd_insert(w.centers[n:n + 1], w.radii[n:n + 1])
        got = collect(ctx)
        want = collect(build_workload(_sub(w, np.arange(n + 1)), precision=precision))
        _same(got, want, n)
        assert 0 < got["stats"]["update_tets"] < w.nt
        assert want["stats"]["update_tets"] == w.nt


def test_insert_many_on_block_equals_fresh_build():
    w = block_c2(h=0.15, ns=300)
    ctx = build_workload(_sub(w, np.arange(260)), precision="fp32")
    ctx.rpd_insert(w.centers[260:], w.radii[260:])
    got = collect(ctx)
    _same(got, collect(build_workload(w, precision="fp32")), "block")
    assert got["stats"]["update_tets"] < w.nt


def test_insert_rejects_bad_input_and_keeps_the_diagram():
    w = torus_c1()
    ctx = build_workload(_sub(w, np.arange(40)))
    before = collect(ctx)
    with pytest.raises(RpdError) as e:
        ctx.rpd_insert(np.array([[np.nan, 0.0, 0.0]]), np.array([0.3]))
    assert e.value.status == RPD_E_INVALID
    _same(collect(ctx), before, "after rejected insert")
    ctx.rpd_insert(w.centers[40:41], w.radii[40:41])
    _same(collect(ctx), collect(build_workload(_sub(w, np.arange(41)))), "after good insert")


# ---------------------------------------------------------- shrinking
@pytest.mark.parametrize("which", ["torus", "tiny_box"])
def test_shrink_matches_cpu_restatement(which):
    """The torus (thousands of boundary triangles, split over the pin's
    cluster of CTAs) and a tiny box (48 triangles, six per CTA): the parts'
    minimum must be the whole surface's."""
    w = torus_c1() if which == "torus" else tiny("box", 1, 5)
    ctx = build_workload(w)
    tris, ids = boundary_triangles(w)
    q, _, _ = w.ints()
    sc = 1.0 / float(1 << w.grid_bits)
    rng = np.random.default_rng(3)
    pick = rng.choice(len(ids), size=min(24, len(ids)), replace=False)
    pins, nrm = [], []
    for k in pick:
        T = tris[k]
        t, f = int(ids[k]) >> 2, int(ids[k]) & 3
        p = T.mean(axis=0)
        n = np.cross(T[1] - T[0], T[2] - T[0])
        n /= np.linalg.norm(n)
        if n @ (q[w.tets[t, f]] * sc - p) < 0:
            n = -n
        pins.append(p)
        nrm.append(n)
    pins, nrm = np.array(pins), np.array(nrm)
    c, r, it = (x.cpu().numpy() for x in ctx.rpd_shrink(pins, nrm, ids[pick].astype(np.int32)))
    r0 = 2.0 ** (23 - w.grid_bits)
    for j, k in enumerate(pick):
        cc, rr, _ = cpu_shrink(tris, int(k), pins[j], nrm[j], r0)
        assert abs(r[j] - rr) <= 1e-9 * rr, (j, r[j], rr)
        assert np.linalg.norm(c[j] - cc) <= 1e-9 * rr
        assert it[j] >= 2


# --------------------------------------------------------------- pins
def _face_centroid3(q, tets, fid):
    t, f = fid >> 2, fid & 3
    cs = [c for c in range(4) if c != f]
    return sum(q[tets[t, c]].astype(np.int64) for c in cs)


def test_pin_of_euler_failure_is_the_furthest_surface_triangle():
    """Ring torus with one sphere: the RPC has chi = 0 (Sec. 3.3 example);
    every tet is whole in it, so the pin is the boundary triangle furthest
    from the sphere (Sec. 4.1.2), ties to the lowest (tet, face)."""
    w = tiny("ring", 1, 0, spheres=ring_spheres(1))
    ctx = build_workload(w)
    keys, pins, nrm, faces = (x.cpu().numpy() for x in ctx.rpd_pins(1))
    assert keys.tolist() == [[0]]
    q, c, _ = w.ints()
    _, ids = boundary_triangles(w)
    d2 = [int(np.sum((_face_centroid3(q, w.tets, int(i)) - 3 * c[0]) ** 2)) for i in ids]
    best = min(int(i) for i, d in zip(ids, d2) if d == max(d2))
    assert faces.tolist() == [best]
    sc = 1.0 / float(1 << w.grid_bits)
    assert np.allclose(pins[0], _face_centroid3(q, w.tets, best) * sc / 3.0, rtol=0, atol=1e-12)
    assert abs(np.linalg.norm(nrm[0]) - 1) < 1e-12
    for kind in (2, 3):
        assert len(ctx.rpd_pins(kind)[0]) == 0


def test_pin_of_component_failure_lies_on_another_component():
    """Ring torus with two spheres: RPF(0,1) has beta0 = 2 (Sec. 3.3); its pin
    is on a boundary triangle of a tet where both spheres have pieces, in the
    component that does not hold the lowest such tet (Sec. 4.1.1)."""
    w = tiny("ring", 2, 0, spheres=ring_spheres(2))
    ctx = build_workload(w)
    keys, pins, nrm, faces = (x.cpu().numpy() for x in ctx.rpd_pins(2))
    assert keys.tolist() == [[0, 1]] and faces[0] >= 0
    g = collect(ctx)
    both = sorted(set(g["tet"][g["sphere"] == 0]) & set(g["tet"][g["sphere"] == 1]))
    t = int(faces[0]) >> 2
    assert t in both and t != both[0]
    adj = oracle.run(w)["raw"]["adj"]
    assert adj[t, int(faces[0]) & 3] < 0


# ---------------------------------------------------------- repair loop
def _oracle_all_contractible(w, c, r, g):
    fin = Workload(w.name, w.verts, w.tets, c, r, w.grid_bits, w.k, w.precision, w.info)
    o = oracle.run(fin)
    for kind in (1, 2, 3):
        d = o["kinds"][kind]
        assert np.all(d["flag"]), (kind, int((~d["flag"]).sum()))
        gk = g["kinds"][kind]
        assert np.array_equal(gk["keys"], d["keys"].astype(np.int32)), kind
        assert np.array_equal(gk["chi"], d["chi"].astype(np.int32)), kind
        assert np.array_equal(gk["beta0"], d["beta0"].astype(np.int32)), kind


def test_repair_ring_from_one_sphere():
    """Sec. 3.3 / 4.1: one sphere in a solid torus (chi = 0) is repaired into a
    diagram whose every element is contractible."""
    w = tiny("ring", 1, 0, spheres=ring_spheres(1))
    ctx = build_workload(w)
    rounds, inserted, failing = ctx.rpd_repair(32)
    assert failing == 0 and inserted >= 2 and rounds >= 1
    c, r = (x.cpu().numpy() for x in ctx.rpd_spheres())
    fin = tiny("ring", len(r), 0, spheres=(c, r))
    ex = rpd_exact(*from_workload(fin))
    assert all(ex["flag"][k] for k in ex["flag"] if len(k) <= 3)


def test_repair_torus_from_four_spheres():
    w = torus_c1()
    ctx = build_workload(_sub(w, np.arange(0, 64, 16)))
    rounds, inserted, failing = ctx.rpd_repair(64)
    assert failing == 0, (rounds, inserted, failing)
    c, r = (x.cpu().numpy() for x in ctx.rpd_spheres())
    _oracle_all_contractible(w, c, r, collect(ctx))


@pytest.mark.parametrize("genus", [0, 1, 2, 3, 4, 5])
def test_repair_genus_slab(genus):
    """The repair workload (shapes of genus 0-5 from a few near-medial
    spheres), small meshes: every element contractible at the end, as judged
    by the oracle on the final sphere set."""
    w = genus_slab(genus, h=0.15, ns=64)
    ctx = build_workload(w)
    rounds, inserted, failing = ctx.rpd_repair(96)
    assert failing == 0, (genus, rounds, inserted, failing)
    c, r = (x.cpu().numpy() for x in ctx.rpd_spheres())
    _oracle_all_contractible(w, c, r, collect(ctx))


@pytest.mark.parametrize("genus", [0, 1, 2, 3, 4, 5])
def test_repair_genus_slab_full_size(genus):
    """The repair workload at its full size (~125k tets, 256 near-medial
    starting spheres): every element contractible at the end, judged by the
    C oracle's same-algorithm tier (kNN candidates, exact predicates; equal
    to its brute force by the CPU tests) on the final sphere set."""
    w = genus_slab(genus, seed=20240330 + 100 + genus, h=0.075, ns=256)
    ctx = build_workload(w)
    rounds, inserted, failing = ctx.rpd_repair(96)
    assert failing == 0, (genus, rounds, inserted, failing)
    c, r = (x.cpu().numpy() for x in ctx.rpd_spheres())
    fin = Workload(w.name, w.verts, w.tets, c, r, w.grid_bits, w.k, w.precision, w.info)
    o = oracle.run(fin, k=32)
    g = collect(ctx)
    for kind in (1, 2, 3):
        d = o["kinds"][kind]
        assert np.all(d["flag"]), (kind, int((~d["flag"]).sum()))
        assert np.array_equal(g["kinds"][kind]["keys"], d["keys"].astype(np.int32)), kind
        assert np.array_equal(g["kinds"][kind]["chi"], d["chi"].astype(np.int32)), kind
        assert np.array_equal(g["kinds"][kind]["beta0"], d["beta0"].astype(np.int32)), kind
