"""GPU library vs the CPU oracle (parity), through the C-ABI.

Bar: bit-exact combinatorics (pieces, element keys, chi, beta0, flags); piece
volumes within 1e-9 vol(t) and first moments (about the tet centroid) within
1e-9 vol(t) diam(t).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.tiny import rpd_exact, from_workload
from paper_2403_18761_gb300 import build_workload, rpd_build, RpdError
from paper_2403_18761_gb300.rpd import collect, RPD_E_INVALID, RPD_E_NONMANIFOLD, RPD_E_DEGENERATE
from rpd_inputs import tiny_set, torus_c1, block_c2, tiny, ring_spheres

pytestmark = pytest.mark.gpu

VOL_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    oracle.build()


def _tet_geometry(w):
    q, _, _ = w.ints()
    s = 1.0 / float(1 << w.grid_bits)
    P = q[w.tets.astype(np.int64)].astype(np.float64) * s
    a, b, c = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    cen = P.mean(axis=1)
    diam = np.max(np.linalg.norm(P[:, :, None, :] - P[:, None, :, :], axis=-1), axis=(1, 2))
    return vol, cen, diam


def _check_pieces(w, g, o_tet, o_sph, o_vol, o_mom, sel=None):
    gt, gs, gv, gm = g["tet"], g["sphere"], g["vol"], g["moment"]
    if sel is not None:
        keep = np.isin(gt, sel)
        gt, gs, gv, gm = gt[keep], gs[keep], gv[keep], gm[keep]
    assert np.array_equal(gt, o_tet) and np.array_equal(gs, o_sph), "piece sets differ"
    vol, cen, diam = _tet_geometry(w)
    vt, ct, dt = vol[gt], cen[gt], diam[gt]
    ev = np.abs(gv - o_vol) / vt
    em = np.linalg.norm((gm - gv[:, None] * ct) - (o_mom - o_vol[:, None] * ct), axis=1) / (vt * dt)
    assert ev.max(initial=0) <= VOL_TOL, ev.max()
    assert em.max(initial=0) <= VOL_TOL, em.max()
    return ev.max(initial=0), em.max(initial=0)


def _check_kinds(g, want):
    for kind in (1, 2, 3, 4):
        gk = g["kinds"][kind]
        wk = want[kind]
        assert np.array_equal(gk["keys"], wk["keys"]), f"kind {kind}: keys differ"
        assert np.array_equal(gk["chi"], wk["chi"]), f"kind {kind}: chi differs"
        assert np.array_equal(gk["beta0"], wk["beta0"]), f"kind {kind}: beta0 differs"
        assert np.array_equal(gk["flag"].astype(bool), wk["flag"]), f"kind {kind}: flags differ"


def _exact_as_kinds(ex):
    out = {}
    for kind in (1, 2, 3, 4):
        ks = sorted(k for k in ex["chi"] if len(k) == kind)
        out[kind] = dict(keys=np.array(ks, dtype=np.int32).reshape(-1, kind),
                         chi=np.array([int(ex["chi"][k]) for k in ks], dtype=np.int32),
                         beta0=np.array([ex["beta0"][k] for k in ks], dtype=np.int32),
                         flag=np.array([ex["flag"][k] for k in ks], dtype=bool))
    return out


# ------------------------------------------------------------ tiny, exact
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("idx", range(12))
def test_tiny_matches_exact_oracle(idx, precision):
    w = tiny_set(12)[idx]
    ex = rpd_exact(*from_workload(w))
    g = collect(build_workload(w, precision=precision))
    keys = sorted(ex["pieces"])
    s = 1.0 / float(1 << w.grid_bits)
    o_tet = np.array([k[0] for k in keys], dtype=np.int32)
    o_sph = np.array([k[1] for k in keys], dtype=np.int32)
    o_vol = np.array([float(ex["pieces"][k][0]) for k in keys]) * s ** 3
    o_mom = np.array([[float(x) for x in ex["pieces"][k][1]] for k in keys]).reshape(-1, 3) * s ** 4
    _check_pieces(w, g, o_tet, o_sph, o_vol, o_mom)
    _check_kinds(g, _exact_as_kinds(ex))


def test_torus_nerve_example_on_gpu():
    """Sec. 3.3 torus example, computed by the library."""
    for n, rpf_b0 in ((1, None), (2, 2), (3, 1)):
        g = collect(build_workload(tiny("ring", n, 0, spheres=ring_spheres(n))))
        cells = g["kinds"][1]
        if n == 1:
            assert cells["chi"].tolist() == [0] and cells["beta0"].tolist() == [1]
        else:
            assert set(cells["chi"].tolist()) == {1} and set(cells["beta0"].tolist()) == {1}
            assert g["kinds"][2]["beta0"].max() == rpf_b0
        if n == 3:
            assert len(g["kinds"][3]["keys"]) == 0


# ------------------------------------------------------ full oracle runs
def _oracle_kinds(o):
    return {k: dict(keys=d["keys"].astype(np.int32), chi=d["chi"].astype(np.int32),
                    beta0=d["beta0"].astype(np.int32), flag=d["flag"]) for k, d in o["kinds"].items()}


@pytest.fixture(scope="module")
def torus():
    w = torus_c1()
    return w, oracle.run(w)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_torus_c1_full_parity(torus, precision):
    w, o = torus
    g = collect(build_workload(w, precision=precision))
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"])
    _check_kinds(g, _oracle_kinds(o))


@pytest.fixture(scope="module")
def block_small():
    w = block_c2(h=0.15, ns=300)
    return w, oracle.run(w)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_block_small_full_parity(block_small, precision):
    w, o = block_small
    g = collect(build_workload(w, precision=precision))
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"])
    _check_kinds(g, _oracle_kinds(o))


@pytest.mark.parametrize("force", [1, 2])
def test_forced_slow_paths_agree(block_small, force):
    """Every non-corner predicate through FP64 (1) or exact integers (2)."""
    w, o = block_small
    g = collect(build_workload(w, precision="fp32", debug=force))
    st = g["stats"]
    assert st["pred_fast"] == 0
    if force == 1:
        assert st["pred_fp64"] > 0
    else:
        assert st["pred_fp64"] == 0 and st["pred_exact"] > 0
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"])
    _check_kinds(g, _oracle_kinds(o))


def test_two_word_neighbour_heap_agrees(block_small):
    """The tiled neighbour search with two-word heap entries (the form used
    above 2^17 spheres) gives the same lists as the warp form with packed
    keys, hence identical results."""
    w, o = block_small
    g = collect(build_workload(w, precision="fp32", debug=4))
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"])
    _check_kinds(g, _oracle_kinds(o))
    h = collect(build_workload(w, precision="fp32"))
    for f in ("tet", "sphere", "vol", "moment"):
        assert np.array_equal(g[f], h[f]), f
    assert g["stats"]["n_pairs"] == h["stats"]["n_pairs"]


def test_export_views_match_per_kind_entry_points(block_small):
    """The binding's queries (views of one rpd_export buffer) hold exactly
    what rpd_euler / rpd_components / rpd_contractible copy out one by one."""
    w, _ = block_small
    ctx = build_workload(w, precision="fp32")
    for kind in (1, 2, 3, 4):
        for name, view in (("rpd_euler", ctx.rpd_euler), ("rpd_components", ctx.rpd_components),
                           ("rpd_contractible", ctx.rpd_contractible)):
            k1, v1 = view(kind)
            k2, v2 = ctx.rows_direct(name, kind)
            assert k1.shape == k2.shape and k1.shape[0] > 0
            assert torch.equal(k1, k2) and torch.equal(v1, v2) and v1.dtype == v2.dtype, (name, kind)
    host, nbytes = ctx.tables_host()   # one copy of the export buffer
    assert nbytes > 0 and sorted(host) == [1, 2, 3, 4]
    for kind in (1, 2, 3, 4):
        keys, chi = ctx.rpd_euler(kind)
        _, beta = ctx.rpd_components(kind)
        _, flag = ctx.rpd_contractible(kind)
        for got, want in zip(host[kind], (keys, chi, beta, flag)):
            assert np.array_equal(got, want.cpu().numpy()), kind
    with pytest.raises(RpdError) as e:
        ctx.rpd_euler(5)
    assert e.value.status == RPD_E_INVALID


def test_k1_uses_candidate_fallback(torus):
    w, o = torus
    g = collect(build_workload(w, k=1))
    assert g["stats"]["cand_fallback"] > 0
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"])
    _check_kinds(g, _oracle_kinds(o))


def test_k1_fallback_on_block_matches_oracle(block_small):
    """k = 1 sends the 13k-tet block's tets that straddle cells through the candidate
    fallback (one block per tet scanning the whole sphere grid); the results
    still match the oracle exactly."""
    w, o = block_small
    g = collect(build_workload(w, precision="fp32", k=1))
    assert g["stats"]["cand_fallback"] > 0
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"])
    _check_kinds(g, _oracle_kinds(o))


# ------------------------------------------------- full size (block, C2)
@pytest.fixture(scope="module")
def block_full():
    w = block_c2()
    return w, collect(build_workload(w, precision="fp32"))


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    return np.load(path)


def test_block_c2_full_matches_stored_oracle(block_full):
    """The whole block workload against the brute-force oracle's stored
    results (tests/golden/make_golden.py): every element table bit for bit,
    the complete piece list, and the volume and first moment of every
    restricted power cell within 1e-9 of its volume (moments: x the mesh
    diameter)."""
    import hashlib
    w, g = block_full
    ref = _golden("block_c2_full.npz")
    h = hashlib.sha256()
    for a in (w.verts, w.tets, w.centers, w.radii):
        h.update(np.ascontiguousarray(a).tobytes())
    assert h.hexdigest() == str(ref["input_digest"]), "the block generator changed: rerun make_golden.py"
    p = hashlib.sha256()
    p.update(np.ascontiguousarray(g["tet"], dtype=np.int32).tobytes())
    p.update(np.ascontiguousarray(g["sphere"], dtype=np.int32).tobytes())
    assert len(g["tet"]) == int(ref["n_pieces"]) and p.hexdigest() == str(ref["pieces_digest"])
    for kind in (1, 2, 3, 4):
        gk = g["kinds"][kind]
        assert np.array_equal(gk["keys"], ref[f"keys{kind}"]), kind
        assert np.array_equal(gk["chi"], ref[f"chi{kind}"]), kind
        assert np.array_equal(gk["beta0"], ref[f"beta{kind}"]), kind
        want_flag = (ref[f"beta{kind}"] == 1) & (ref[f"chi{kind}"] == 1)
        assert np.array_equal(gk["flag"].astype(bool), want_flag), kind
    cv = np.bincount(g["sphere"], weights=g["vol"], minlength=w.ns)
    vref = ref["cell_vol"]
    assert np.all(np.abs(cv - vref) <= 1e-9 * vref)
    diam = float(np.linalg.norm(w.verts.max(axis=0) - w.verts.min(axis=0)))
    for a in range(3):
        cm = np.bincount(g["sphere"], weights=g["moment"][:, a], minlength=w.ns)
        assert np.all(np.abs(cm - ref[f"cell_mom{a}"]) <= 1e-9 * vref * diam), a


def test_block_c2_sampled_tets_match_oracle(block_full):
    w, g = block_full
    rng = np.random.default_rng(7)
    sub = np.sort(rng.choice(w.nt, size=2000, replace=False)).astype(np.int32)
    o = oracle.run(w, subset=sub)
    _check_pieces(w, g, o["tet"], o["sphere"], o["vol"], o["moment"], sel=sub)


def test_block_c2_invariants(block_full):
    w, g = block_full
    vol, _, _ = _tet_geometry(w)
    per = np.bincount(g["tet"], weights=g["vol"], minlength=w.nt)
    assert np.all(np.abs(per - vol) <= 1e-12 * vol)
    tot = sum((-1) ** (k - 1) * int(d["chi"].sum()) for k, d in g["kinds"].items())
    assert tot == w.info["chi"] == -2
    for d in g["kinds"].values():
        k = d["keys"]
        assert np.all(np.diff(k, axis=1) > 0) if k.shape[1] > 1 else True
        assert np.all(d["beta0"] >= 1)
        assert np.array_equal(d["flag"].astype(bool), (d["beta0"] == 1) & (d["chi"] == 1))


def test_block_c2_precisions_and_runs_agree(block_full):
    w, g = block_full
    h = collect(build_workload(w, precision="fp64"))
    g2 = collect(build_workload(w, precision="fp32"))
    for other in (h, g2):
        assert np.array_equal(other["tet"], g["tet"]) and np.array_equal(other["sphere"], g["sphere"])
        for kind in (1, 2, 3, 4):
            for f in ("keys", "chi", "beta0", "flag"):
                assert np.array_equal(other["kinds"][kind][f], g["kinds"][kind][f])
    assert np.array_equal(g2["vol"], g["vol"])
    assert np.max(np.abs(h["vol"] - g["vol"])) <= 1e-12 * np.max(g["vol"])


# ---------------------------------------------------------- error paths
def test_rejects_inverted_tet():
    w = tiny("block", 3, 1)
    t = w.tets.copy()
    t[0, [2, 3]] = t[0, [3, 2]]
    with pytest.raises(RpdError) as e:
        rpd_build(w.verts, t, w.centers, w.radii, grid_bits=w.grid_bits)
    assert e.value.status == RPD_E_INVALID


def test_rejects_nan_and_out_of_range():
    w = tiny("block", 3, 1)
    v = w.verts.copy()
    v[0, 0] = np.nan
    with pytest.raises(RpdError) as e:
        rpd_build(v, w.tets, w.centers, w.radii, grid_bits=w.grid_bits)
    assert e.value.status == RPD_E_INVALID
    with pytest.raises(RpdError) as e:
        rpd_build(w.verts * 1e6, w.tets, w.centers, w.radii, grid_bits=w.grid_bits)
    assert e.value.status == RPD_E_INVALID


def test_rejects_face_shared_by_three_tets():
    w = tiny("block", 3, 1)
    t = np.concatenate([w.tets, w.tets[:1]], axis=0)
    with pytest.raises(RpdError) as e:
        rpd_build(w.verts, t, w.centers, w.radii, grid_bits=w.grid_bits)
    assert e.value.status == RPD_E_NONMANIFOLD


def test_reports_degenerate_input():
    """A mesh vertex exactly on the radical plane of two equal spheres."""
    w = tiny("box", 2, 5)
    s = 1.0 / float(1 << w.grid_bits)
    v = w.verts[w.tets[0, 0]]
    d = np.array([5.0, 3.0, 1.0]) * 1024 * s
    c = np.stack([v + d, v - d])
    with pytest.raises(RpdError) as e:
        rpd_build(w.verts, w.tets, c, np.full(2, 2048 * s), grid_bits=w.grid_bits)
    assert e.value.status == RPD_E_DEGENERATE
