"""The same-algorithm CPU baseline (oracle.run(w, k=K): the library's neighbour
+ candidate algorithm restated in C, clipping each candidate by the other
candidates only) gives exactly the brute force's pieces and elements.  Its
pin is the brute force itself: clipping by every sphere (Eq. 1-3) must give
the same pieces as clipping by any superset of the spheres whose cells meet
the tet, and k = 1 forces the scan taken when the neighbour lists do not
cover a tet's thresholds."""
import numpy as np
import pytest

import oracle
from rpd_inputs import torus_c1, block_c2


@pytest.fixture(scope="module")
def cases():
    oracle.build()
    out = []
    for w in (torus_c1(), block_c2(h=0.15, ns=300)):
        out.append((w, oracle.run(w)))
    return out


@pytest.mark.parametrize("k", [1, 4, 32])
def test_same_algorithm_equals_brute_force(cases, k):
    for w, brute in cases:
        fair = oracle.run(w, k=min(k, 32))
        assert np.array_equal(fair["tet"], brute["tet"]) and np.array_equal(fair["sphere"], brute["sphere"])
        assert np.max(np.abs(fair["vol"] - brute["vol"])) <= 1e-12 * np.max(brute["vol"])
        for kind in (1, 2, 3, 4):
            for f in ("keys", "chi", "beta0"):
                assert np.array_equal(fair["kinds"][kind][f], brute["kinds"][kind][f]), (w.name, k, kind, f)


def test_same_algorithm_on_a_subset(cases):
    w, brute = cases[1]
    rng = np.random.default_rng(5)
    sub = np.sort(rng.choice(w.nt, size=500, replace=False)).astype(np.int32)
    a = oracle.run(w, subset=sub)
    b = oracle.run(w, subset=sub, k=w.k)
    assert np.array_equal(a["tet"], b["tet"]) and np.array_equal(a["sphere"], b["sphere"])
    assert np.array_equal(a["vol"], b["vol"])
