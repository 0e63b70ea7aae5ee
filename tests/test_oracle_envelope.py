"""The CPU envelope distance (oracle/envelope.py, Sec. 4.3) against closed
forms: spheres, capsules (cones with equal radii), thickened triangles (slabs
with equal radii) and the tangent-angle solution of a cone with growing
radius."""
import numpy as np

from oracle.envelope import cone_distance, slab_distance, envelope_distance


def _seg_dist(s, a, b):
    t = np.clip(np.einsum("ij,j->i", s - a, b - a) / np.dot(b - a, b - a), 0, 1)
    return np.linalg.norm(s - (a + t[:, None] * (b - a)), axis=1)


def _tri_dist(s, A, B, C):
    n = np.cross(B - A, C - A)
    n /= np.linalg.norm(n)
    h = (s - A) @ n
    p = s - h[:, None] * n
    inside = np.ones(len(s), bool)
    for U, V in ((A, B), (B, C), (C, A)):
        inside &= np.cross(V - U, p - U) @ n >= 0
    d = np.where(inside, np.abs(h), np.inf)
    for U, V in ((A, B), (B, C), (C, A)):
        d = np.minimum(d, _seg_dist(s, U, V))
    return d


def test_capsule_and_thick_triangle():
    rng = np.random.default_rng(1)
    S = rng.uniform(-2, 2, (200, 3))
    a, b = np.array([0.1, -0.3, 0.2]), np.array([1.2, 0.7, -0.4])
    got = cone_distance(S, a[None], np.array([0.3]), b[None], np.array([0.3]))[:, 0]
    assert np.allclose(got, _seg_dist(S, a, b) - 0.3, atol=1e-9)
    A, B, C = np.array([0.0, 0, 0]), np.array([1.0, 0.2, 0]), np.array([0.3, 1.1, 0.4])
    got = slab_distance(S, A[None], np.array([0.25]), B[None], np.array([0.25]), C[None], np.array([0.25]))[:, 0]
    assert np.allclose(got, _tri_dist(S, A, B, C) - 0.25, atol=1e-8)


def test_cone_tangent_angle():
    """Cone along x from (0,0,0) r=0.2 to (2,0,0) r=0.6 (slope k = 0.2): for a
    point at axial x and radial y whose stationary point z = x + k y /
    sqrt(1 - k^2) lies in (0, 2), the distance is y sqrt(1 - k^2) - (r1 + k x)."""
    k = 0.2
    S = np.array([[0.9, 1.0, 0.0], [1.1, 0.0, 1.5], [0.5, -0.8, 0.6]])
    got = cone_distance(S, np.zeros((1, 3)), np.array([0.2]), np.array([[2.0, 0, 0]]), np.array([0.6]))[:, 0]
    x = S[:, 0]
    y = np.hypot(S[:, 1], S[:, 2])
    z = x + k * y / np.sqrt(1 - k * k)
    assert np.all((z > 0) & (z < 2))
    want = y * np.sqrt(1 - k * k) - (0.2 + k * x)
    assert np.allclose(got, want, atol=1e-9)


def test_envelope_is_minimum_over_primitives():
    C = np.array([[0.0, 0, 0], [2.0, 0, 0], [1.0, 1.5, 0]])
    R = np.array([0.5, 0.4, 0.3])
    S = np.array([[1.0, -1.0, 0.0], [5.0, 5.0, 5.0], [1.0, 0.5, 2.0]])
    d0 = envelope_distance(S, C, R, [], [])
    d1 = envelope_distance(S, C, R, [(0, 1), (0, 2), (1, 2)], [])
    d2 = envelope_distance(S, C, R, [(0, 1), (0, 2), (1, 2)], [(0, 1, 2)])
    assert np.all(d1 <= d0 + 1e-12) and np.all(d2 <= d1 + 1e-12)
    assert d2[0] < d0[0]   # below the base, the cone/slab is closer than the spheres
