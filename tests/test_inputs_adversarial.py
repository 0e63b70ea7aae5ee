"""The near-degenerate generators produce what they claim, checked with exact
rationals: the point where two radical planes meet a mesh edge (or a mesh
corner) is off the third plane by a nonzero amount of at most one squared grid
unit, and the exact oracle runs on them without meeting a zero sign."""
from fractions import Fraction

import pytest

from oracle.tiny import rpd_exact, from_workload
from rpd_inputs.adversarial import near_edge_triple, near_corner, near_parallel


def _pd(x, c, w):
    return sum((Fraction(a) - b) ** 2 for a, b in zip(x, c)) - w


def _ints(w):
    q, c, r = w.ints()
    return ([tuple(int(v) for v in row) for row in q], [tuple(int(v) for v in row) for row in c],
            [int(v) * int(v) for v in r])


@pytest.mark.parametrize("seed", [1, 2])
def test_near_edge_triple(seed):
    w = near_edge_triple(seed)
    _, C, W = _ints(w)
    X0, X1 = w.info["edge"]
    t = w.info["crossing"]
    P = tuple(Fraction(a) + t * (b - a) for a, b in zip(X0, X1))
    assert _pd(P, C[0], W[0]) == _pd(P, C[1], W[1])          # on the (0, 1) radical plane
    miss = _pd(P, C[0], W[0]) - _pd(P, C[2], W[2])            # off the (0, 2) plane
    assert miss == w.info["miss"] and 0 < abs(miss) <= 1
    ex = rpd_exact(*from_workload(w))
    assert any(len(k) == 3 for k in ex["chi"])                # the three cells meet


@pytest.mark.parametrize("sign", [1, -1])
def test_near_corner(sign):
    w = near_corner(1, sign)
    _, C, W = _ints(w)
    X = w.info["corner"]
    assert _pd(X, C[0], W[0]) - _pd(X, C[1], W[1]) == sign
    rpd_exact(*from_workload(w))


def test_near_parallel():
    w = near_parallel(1)
    _, C, W = _ints(w)
    a = [cj - ci for ci, cj in zip(C[0], C[1])]
    b = [ck - ci for ci, ck in zip(C[0], C[2])]
    cr = (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])
    # centres almost collinear: the radical-plane normals c_j - c_i and c_k - c_i
    # make an angle below 1e-4 rad
    sin2 = Fraction(sum(v * v for v in cr), sum(v * v for v in a) * sum(v * v for v in b))
    assert sin2 < Fraction(1, 10 ** 8)
    assert abs(w.info["miss"]) <= 1 and w.info["miss"] != 0
    ex = rpd_exact(*from_workload(w))
    assert any(len(k) == 3 for k in ex["chi"])
