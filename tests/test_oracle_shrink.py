"""The CPU restatement of sphere shrinking (oracle/shrink.py, Sec. 5.1) against
closed forms: the largest ball tangent at a boundary point inside a closed
convex polyhedron, and emptiness / two-point tangency on a non-convex mesh."""
import numpy as np
import pytest

from oracle.shrink import shrink, nearest_points, boundary_triangles
from rpd_inputs import tiny


def _icosphere(level):
    t = (1 + 5 ** 0.5) / 2
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        mid = {}
        F2 = []
        for a, b, c in F:
            m = []
            for u, v in ((a, b), (b, c), (c, a)):
                k = (min(u, v), max(u, v))
                if k not in mid:
                    x = V[u] + V[v]
                    V.append(x / np.linalg.norm(x))
                    mid[k] = len(V) - 1
                m.append(mid[k])
            F2 += [(a, m[0], m[2]), (b, m[1], m[0]), (c, m[2], m[1]), (m[0], m[1], m[2])]
        F = F2
    V = np.array(V)
    return np.array([[V[a], V[b], V[c]] for a, b, c in F])


def _box(a, b, c):
    P = np.array([[x, y, z] for x in (-a, a) for y in (-b, b) for z in (-c, c)])
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    tris = []
    for q in quads:
        tris.append([P[q[0]], P[q[1]], P[q[2]]])
        tris.append([P[q[0]], P[q[2]], P[q[3]]])
    return np.array(tris, float)


def _convex_radius(tris, own, p, m):
    """min_j (d_j - n_j.p) / (1 + n_j.m) over the face planes (outward n_j)."""
    cen = tris.reshape(-1, 3).mean(axis=0)
    best = np.inf
    for j, T in enumerate(tris):
        if j == own:
            continue
        n = np.cross(T[1] - T[0], T[2] - T[0])
        n /= np.linalg.norm(n)
        if n @ (T[0] - cen) < 0:
            n = -n
        den = 1 + n @ m
        if den > 1e-12:
            best = min(best, (n @ T[0] - n @ p) / den)
    return best


def _inward(T, cen):
    n = np.cross(T[1] - T[0], T[2] - T[0])
    n /= np.linalg.norm(n)
    return -n if n @ (T[0] - cen) > 0 else n


@pytest.mark.parametrize("shape", ["box", "icosphere"])
def test_largest_tangent_ball_in_convex_polyhedron(shape):
    tris = _box(2.0, 1.0, 0.5) if shape == "box" else _icosphere(2)
    cen = tris.reshape(-1, 3).mean(axis=0)
    rng = np.random.default_rng(1)
    for own in rng.choice(len(tris), size=6, replace=False):
        T = tris[own]
        p = T.mean(axis=0)
        m = _inward(T, cen)
        c, r, it = shrink(tris, int(own), p, m, 100.0)
        want = _convex_radius(tris, int(own), p, m)
        assert abs(r - want) <= 1e-9 * want, (shape, own, r, want, it)
        assert np.allclose(c, p + r * m)


def test_nearest_point_on_triangle_closed_forms():
    T = np.array([[[0.0, 0, 0], [1, 0, 0], [0, 1, 0]]])
    for x, q in (((0.2, 0.2, 5.0), (0.2, 0.2, 0)), ((-1.0, -1, 0), (0, 0, 0)), ((2.0, -1, 3), (1, 0, 0)),
                 ((0.5, -2, 0), (0.5, 0, 0)), ((1.0, 1, 0), (0.5, 0.5, 0)), ((-3.0, 0.25, 1), (0, 0.25, 0))):
        assert np.allclose(nearest_points(T, np.array(x))[0], q)


def test_ball_on_nonconvex_mesh_is_empty_and_touches_twice():
    w = tiny("ring", 1, 0)
    tris, ids = boundary_triangles(w)
    q, _, _ = w.ints()
    sc = 1.0 / float(1 << w.grid_bits)
    for own in (0, 7, 20, 33):
        T = tris[own]
        p = T.mean(axis=0)
        t, f = int(ids[own]) >> 2, int(ids[own]) & 3
        opposite = q[w.tets[t, f]] * sc            # the tet's corner off this face: inside
        n = np.cross(T[1] - T[0], T[2] - T[0])
        n /= np.linalg.norm(n)
        m = n if n @ (opposite - p) > 0 else -n
        c, r, _ = shrink(tris, own, p, m, 50.0)
        rest = np.delete(tris, own, 0)
        qq = nearest_points(rest, c)
        d = np.sqrt(np.min(np.einsum("ij,ij->i", qq - c, qq - c)))
        assert d >= r * (1 - 1e-9)          # empty
        assert abs(d - r) <= 1e-9 * r       # touches the surface at a second point
        assert r < 3.0                      # bounded by the shape
