"""Near-degenerate sphere sets on the tiny meshes (input generator only).

Generic seeded inputs keep every clipping predicate far from zero, so a
floating-point filter certifies them all.  These generators place spheres so
that a point of the restricted power diagram lies within about one squared
grid unit of another radical plane, while staying in general position
(nothing exactly on a plane):

* ``near_edge_triple``  three spheres whose common radical line crosses a
  mesh edge: the crossing point of two of the radical planes with the edge is
  off the third plane by |r_k^2 - w*| <= 1 grid unit^2;
* ``near_corner``       a mesh corner off the radical plane of two spheres by
  exactly +1 or -1 grid unit^2 of power;
* ``near_parallel``     two radical planes of one sphere that nearly coincide
  (centres almost collinear) and cross inside a tet.

Everything is integer or rational geometry on the grid (squared distances of
points and the crossing point of a plane with an edge); the construction
holds none of the restricted-power-diagram method.  Results are Workloads on
the integer grid, like the rest of this package.
"""
from __future__ import annotations

from fractions import Fraction
from math import isqrt, lcm

import numpy as np

from .configs import tiny


def _d2(p, c):
    return sum((a - b) ** 2 for a, b in zip(p, c))


def _finish(w0, cs, rs):
    s = 1.0 / float(1 << w0.grid_bits)
    c = np.array(cs, dtype=np.float64) * s
    r = np.array(rs, dtype=np.float64) * s
    return tiny("box", len(rs), int(w0.info.get("seed", 0)), spheres=(c, r))


def _mesh(seed):
    w0 = tiny("box", 1, seed)
    w0.info["seed"] = seed
    q, _, _ = w0.ints()
    return w0, [tuple(int(v) for v in row) for row in q]


def _interior_edge(w0, q, rng):
    """An edge of a tet near the middle of the box: (X0, X1) as int tuples."""
    cen = np.array(q, dtype=np.float64).mean(axis=0)
    tc = np.array(q, dtype=np.float64)[w0.tets].mean(axis=1)
    order = np.argsort(np.linalg.norm(tc - cen, axis=1))
    t = int(order[int(rng.integers(0, 6))])
    a, b = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)][int(rng.integers(0, 6))]
    return q[int(w0.tets[t, a])], q[int(w0.tets[t, b])]


def _rand_centre(rng, m, spread):
    return tuple(int(v) for v in np.rint(np.asarray(m, dtype=np.float64) + rng.uniform(-spread, spread, 3)))


def _centres(rng, m, spread, n, batch=4096):
    """n random integer points in the box m +- spread, drawn in batches."""
    m = np.asarray(m, dtype=np.float64)
    while n > 0:
        b = min(batch, n)
        for row in np.rint(m + rng.uniform(-spread, spread, (b, 3))).astype(np.int64).tolist():
            yield tuple(row)
        n -= b


def _square_near(P, base, centres):
    """First (c, r, miss) among `centres` with 0 < |r^2 - w*| <= 1, where
    w* = |P - c|^2 + base, P a rational point and base rational; integer
    arithmetic on a common denominator."""
    den = 1
    for v in P:
        den = lcm(den, Fraction(v).denominator)
    Pn = [int(Fraction(v) * den) for v in P]
    d2 = den * den
    B = Fraction(base) * d2
    assert B.denominator == 1
    B = B.numerator
    for c in centres:
        N = sum((pn - den * ci) ** 2 for pn, ci in zip(Pn, c)) + B   # w* = N / den^2
        if N <= 0:
            continue
        r0 = isqrt(N // d2)
        for r in (r0, r0 + 1):
            dn = r * r * d2 - N
            if dn != 0 and abs(dn) <= d2:
                return c, r, Fraction(dn, d2)
    return None


def near_edge_triple(seed: int, max_trials: int = 400000):
    """Three spheres i, j, k: the radical plane of (i, j) crosses a mesh edge at
    P, and the radical plane of (i, k) misses P by |r_k^2 - w*| <= 1 grid
    unit^2 of power (w* = the weight that would put P exactly on it)."""
    rng = np.random.default_rng(seed)
    w0, q = _mesh(seed)
    S = 1 << w0.grid_bits
    X0, X1 = _interior_edge(w0, q, rng)
    M = tuple((a + b) / 2 for a, b in zip(X0, X1))
    for _ in range(100):
        ci = _rand_centre(rng, M, 0.8 * S)
        ri = int(rng.integers(int(0.3 * S), int(0.6 * S)))
        cj = _rand_centre(rng, M, 0.8 * S)
        t0 = float(rng.uniform(0.3, 0.7))
        P0 = tuple(int(round(a + t0 * (b - a))) for a, b in zip(X0, X1))
        wj = _d2(P0, cj) - _d2(P0, ci) + ri * ri
        if wj <= 0:
            continue
        rj = isqrt(wj)
        # exact crossing of the (i, j) radical plane with the edge
        f0 = _d2(X0, ci) - ri * ri - _d2(X0, cj) + rj * rj
        f1 = _d2(X1, ci) - ri * ri - _d2(X1, cj) + rj * rj
        if f0 == f1 or (f0 > 0) == (f1 > 0) or f0 == 0 or f1 == 0:
            continue
        t = Fraction(f0, f0 - f1)
        if not (Fraction(1, 5) < t < Fraction(4, 5)):
            continue
        P = tuple(a + t * (b - a) for a, b in zip(X0, X1))
        base = -_d2(P, ci) + ri * ri   # w* = |P - c_k|^2 + base
        best = _square_near(P, base, _centres(rng, M, 0.9 * S, max_trials))
        if best and best[1] > S // 8:
            ck, rk, diff = best
            w = _finish(w0, [ci, cj, ck], [ri, rj, rk])
            w.info.update(kind="near_edge_triple", edge=(X0, X1), crossing=t, miss=diff)
            return w
    raise RuntimeError("no near-degenerate triple found")


def near_corner(seed: int, sign: int = 1, max_trials: int = 2000000):
    """Two spheres whose radical plane misses a mesh corner X by exactly
    `sign` grid unit^2 of power: pd(X, i) - pd(X, j) = sign."""
    rng = np.random.default_rng(seed)
    w0, q = _mesh(seed)
    S = 1 << w0.grid_bits
    X0, _ = _interior_edge(w0, q, rng)
    ci = _rand_centre(rng, X0, 0.7 * S)
    ri = int(rng.integers(int(0.3 * S), int(0.6 * S)))
    for cj in _centres(rng, X0, 0.9 * S, max_trials):
        wj = _d2(X0, cj) - _d2(X0, ci) + ri * ri + sign
        if wj <= 0:
            continue
        rj = isqrt(wj)
        if rj * rj == wj:
            w = _finish(w0, [ci, cj], [ri, rj])
            w.info.update(kind="near_corner", corner=X0, miss=sign)
            return w
    raise RuntimeError("no near-corner pair found")


def near_parallel(seed: int, max_trials: int = 400000):
    """Spheres i, j, k with c_k - c_i = 2 (c_j - c_i) + d, |d| = 1 grid unit
    per axis at most, so the radical planes (i, j) and (i, k) are almost
    parallel; the weight of k makes them cross within 1 grid unit^2 of power
    of a point Q on the (i, j) plane inside the mesh."""
    rng = np.random.default_rng(seed)
    w0, q = _mesh(seed)
    S = 1 << w0.grid_bits
    X0, X1 = _interior_edge(w0, q, rng)
    M = tuple((a + b) / 2 for a, b in zip(X0, X1))
    for _ in range(100):
        ci = _rand_centre(rng, M, 0.6 * S)
        ri = int(rng.integers(int(0.3 * S), int(0.5 * S)))
        cj = _rand_centre(rng, M, 0.6 * S)
        P0 = tuple(int(round(a + 0.5 * (b - a))) for a, b in zip(X0, X1))
        wj = _d2(P0, cj) - _d2(P0, ci) + ri * ri
        if wj <= 0:
            continue
        rj = isqrt(wj)
        f0 = _d2(X0, ci) - ri * ri - _d2(X0, cj) + rj * rj
        f1 = _d2(X1, ci) - ri * ri - _d2(X1, cj) + rj * rj
        if f0 == f1 or (f0 > 0) == (f1 > 0) or f0 == 0 or f1 == 0:
            continue
        t = Fraction(f0, f0 - f1)
        Q = tuple(a + t * (b - a) for a, b in zip(X0, X1))
        base = -_d2(Q, ci) + ri * ri

        def centres():
            left = max_trials
            while left > 0:
                nb = min(4096, left)
                left -= nb
                D = rng.integers(-1, 2, (nb, 3)).tolist()
                SH = rng.integers(-S // 8, S // 8, nb).tolist()
                for d, sh in zip(D, SH):
                    if d == [0, 0, 0]:
                        continue
                    # move along the line of centres as well, so the trials differ
                    yield tuple(a + 2 * (b - a) + dd + (sh * (b - a)) // S for a, b, dd in zip(ci, cj, d))
        best = _square_near(Q, base, centres())
        if best:
            ck, rk, diff = best
            w = _finish(w0, [ci, cj, ck], [ri, rj, rk])
            w.info.update(kind="near_parallel", miss=diff)
            return w
    raise RuntimeError("no near-parallel pair found")
