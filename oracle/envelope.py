"""Distance to the medial mesh's enveloping volume on the CPU (TEST
INFRASTRUCTURE ONLY: only tests/ use it).

Sec. 4.3 measures, for every surface sample s, the distance to the closest
enveloping element of the medial mesh: a medial sphere (c, r), a medial cone
(the spheres interpolated linearly between two vertices, Sec. 3.1) or a medial
slab (between three).  Written from that definition: for a primitive with
spheres (c_a, r_a) the distance is the minimum over interpolation weights l
(l >= 0, sum 1) of |s - sum l_a c_a| - sum l_a r_a.  The function is convex in
l, so the minimum is found by golden-section search: over t in [0, 1] for a
cone, nested (outer over l_3, inner over l_2 in [0, 1 - l_3]) for a slab.
No closed form and no code shared with the library.

Pins (tests/test_oracle_envelope.py): a cone with equal radii is a capsule
(distance to the axis segment minus r), a slab with equal radii a thickened
triangle (distance to the triangle minus r), and a cone whose radius grows
with slope k has the closed-form tangent angle.
"""
from __future__ import annotations

import numpy as np

_G = (np.sqrt(5.0) - 1.0) / 2.0


def _golden(f, lo, hi, iters=90):
    """Minimum of convex f over [lo, hi] (arrays), elementwise: the bracket
    [a, b] shrinks by the golden ratio each step, keeping the side of the
    interior point with the smaller value."""
    a, b = lo.astype(np.float64), hi.astype(np.float64)
    c = b - _G * (b - a)
    d = a + _G * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        left = fc < fd                      # minimum in [a, d]
        a, b = np.where(left, a, c), np.where(left, d, b)
        c_new = np.where(left, b - _G * (b - a), d)
        d_new = np.where(left, c, a + _G * (b - a))
        fc, fd = np.where(left, f(c_new), fd), np.where(left, fc, f(d_new))
        c, d = c_new, d_new
    return np.minimum(np.minimum(fc, fd), np.minimum(f(a), f(b)))


def _dist(s, c, r):
    return np.linalg.norm(s - c, axis=-1) - r


def sphere_distance(S, C, R):
    """(n samples, m spheres) distances."""
    return np.linalg.norm(S[:, None, :] - C[None, :, :], axis=-1) - R[None, :]


def cone_distance(S, C1, R1, C2, R2):
    s = S[:, None, :]

    def f(t):
        c = C1[None] + t[..., None] * (C2 - C1)[None]
        return _dist(s, c, R1[None] + t * (R2 - R1)[None])

    shape = (len(S), len(C1))
    return _golden(f, np.zeros(shape), np.ones(shape))


def slab_distance(S, C1, R1, C2, R2, C3, R3, iters=70):
    s = S[:, None, :]
    shape = (len(S), len(C1))

    def inner(l3):
        def f(l2):
            c = C1[None] + l2[..., None] * (C2 - C1)[None] + l3[..., None] * (C3 - C1)[None]
            r = R1[None] + l2 * (R2 - R1)[None] + l3 * (R3 - R1)[None]
            return _dist(s, c, r)
        return _golden(f, np.zeros(shape), 1.0 - l3, iters)

    return _golden(inner, np.zeros(shape), np.ones(shape), iters)


def envelope_distance(S, centres, radii, edges, faces, vertices=None):
    """Distance of samples S (n, 3) to the union of the spheres (the rows
    `vertices` of centres/radii, all rows when None), cones (edges, pairs of
    rows) and slabs (faces, triples of rows): the minimum over all of them."""
    S = np.asarray(S, dtype=np.float64)
    v = np.arange(len(radii)) if vertices is None else np.asarray(vertices)
    best = sphere_distance(S, centres[v], radii[v]).min(axis=1)
    if len(edges):
        e = np.asarray(edges)
        best = np.minimum(best, cone_distance(S, centres[e[:, 0]], radii[e[:, 0]], centres[e[:, 1]],
                                              radii[e[:, 1]]).min(axis=1))
    if len(faces):
        f = np.asarray(faces)
        best = np.minimum(best, slab_distance(S, centres[f[:, 0]], radii[f[:, 0]], centres[f[:, 1]], radii[f[:, 1]],
                                              centres[f[:, 2]], radii[f[:, 2]]).min(axis=1))
    return best
