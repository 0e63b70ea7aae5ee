"""The C brute-force oracle against the exact-rational oracle and invariants."""
import numpy as np
import pytest

import oracle
from oracle.tiny import rpd_exact, from_workload
from rpd_inputs import tiny_set, torus_c1, tiny


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _compare(w, nthreads=2):
    ex = rpd_exact(*from_workload(w))
    o = oracle.run(w, nthreads=nthreads)
    s = 1.0 / float(1 << w.grid_bits)
    keys = sorted(ex["pieces"])
    assert keys == list(zip(o["tet"].tolist(), o["sphere"].tolist()))
    for k, v, m in zip(keys, o["vol"], o["moment"]):
        ev = float(ex["pieces"][k][0]) * s ** 3
        em = np.array([float(x) for x in ex["pieces"][k][1]]) * s ** 4
        assert abs(v - ev) <= 1e-12 * ev
        assert np.all(np.abs(m - em) <= 1e-12 * np.abs(em).max())
    n = 0
    for kind, d in o["kinds"].items():
        for key, c, cf, b in zip(d["keys"], d["chi"], d["chi_frac"], d["beta0"]):
            kk = tuple(int(x) for x in key)
            assert ex["chi"][kk] == c and abs(cf - c) < 1e-9
            assert ex["beta0"][kk] == b
            n += 1
    assert n == len(ex["chi"])


@pytest.mark.parametrize("idx", range(12))
def test_c_oracle_matches_exact_oracle(idx):
    _compare(tiny_set(12)[idx])


def test_c_oracle_thread_count_does_not_matter():
    w = tiny_set(3)[1]
    a, b = oracle.run(w, nthreads=1), oracle.run(w, nthreads=3)
    assert np.array_equal(a["tet"], b["tet"]) and np.array_equal(a["vol"], b["vol"])


def _mesh_volume(w):
    q, _, _ = w.ints()
    P = q[w.tets.astype(np.int64)]
    a, b, c = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]
    det = np.einsum("ij,ij->i", a, np.cross(b, c))       # exact in int64 (short edges)
    s = 1.0 / float(1 << w.grid_bits)
    vol = det.astype(np.float64) / 6.0 * s ** 3
    cen = P.sum(axis=1).astype(np.float64) / 4.0 * s
    return vol, cen


@pytest.fixture(scope="module")
def c1():
    w = torus_c1()
    return w, oracle.run(w)


def test_c1_volumes_partition_the_mesh(c1):
    w, o = c1
    vol, cen = _mesh_volume(w)
    per_tet = np.bincount(o["tet"], weights=o["vol"], minlength=w.nt)
    assert np.all(np.abs(per_tet - vol) <= 1e-12 * vol)
    mom = (vol[:, None] * cen)
    got = np.stack([np.bincount(o["tet"], weights=o["moment"][:, k], minlength=w.nt) for k in range(3)], 1)
    assert np.all(np.abs(got - mom) <= 1e-11 * np.abs(mom).max())


def test_c1_inclusion_exclusion(c1):
    w, o = c1
    tot = sum((-1) ** (kind - 1) * int(d["chi"].sum()) for kind, d in o["kinds"].items())
    assert tot == w.info["chi"] == 0


def test_c1_owner_rule_matches_fractional(c1):
    _, o = c1
    for d in o["kinds"].values():
        assert np.all(np.abs(d["chi_frac"] - d["chi"]) < 1e-9)


def test_c1_single_sphere_is_the_torus():
    w = torus_c1()
    w.centers, w.radii = w.centers[:1], w.radii[:1]
    o = oracle.run(w)
    d = o["kinds"][1]
    assert d["chi"].tolist() == [0] and d["beta0"].tolist() == [1]
    assert len(o["tet"]) == w.nt


def test_c1_subset_matches_full(c1):
    w, o = c1
    sub = np.arange(0, w.nt, 37, dtype=np.int32)
    s = oracle.run(w, subset=sub)
    sel = np.isin(o["tet"], sub)
    assert np.array_equal(s["tet"], o["tet"][sel]) and np.array_equal(s["sphere"], o["sphere"][sel])
    assert np.array_equal(s["vol"], o["vol"][sel])
