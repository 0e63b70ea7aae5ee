"""Sphere shrinking on the CPU (TEST INFRASTRUCTURE ONLY: only tests/ use it).

Sec. 5.1 computes medial spheres tangent to two surface points with the
shrinking-ball algorithm (Ma et al. 2012): from a pin point p on the surface
with inward unit normal n, start from a ball tangent at p, centre p + r n; take
the surface point q nearest to the centre; if q is inside the ball, replace the
ball by the one tangent at p that passes through q, whose radius solves
|p + r n - q| = r, i.e. r = |p - q|^2 / (2 n.(q - p)); repeat until the ball
contains no surface point.  The surface is a set of triangles; the pin's own
triangle is left out (it touches the ball at p).

Nearest point on a triangle, written from its definition: the orthogonal
projection onto the triangle's plane when its barycentric coordinates
(ratios of sub-triangle areas, signed by the plane normal) are all >= 0,
otherwise the nearest of the three edges' nearest points (projection onto the
edge's line clamped to the segment).  Plain numpy over all triangles; no code
is shared with the CUDA library.

The paper cites the algorithm and prints no worked example.  The CPU tests
pin this restatement to closed forms instead: inside a closed convex
polyhedron with face planes n_j.x <= d_j (outward unit n_j), the largest ball
tangent at p with inward normal m has radius min_j (d_j - n_j.p) / (1 + n_j.m)
(checked on a box and on a subdivided icosahedron), and on a non-convex mesh
the final ball is empty and touches the surface at p and at one more point.
"""
from __future__ import annotations

import numpy as np


def _segment_nearest(P, Q, x):
    d = Q - P
    l2 = np.einsum("ij,ij->i", d, d)
    u = np.where(l2 > 0, np.einsum("ij,ij->i", x - P, d) / np.where(l2 > 0, l2, 1.0), 0.0)
    u = np.clip(u, 0.0, 1.0)
    return P + u[:, None] * d


def nearest_points(tris, x):
    """Nearest point of each triangle (m, 3, 3) to the point x (3,): (m, 3)."""
    A, B, C = tris[:, 0], tris[:, 1], tris[:, 2]
    nrm = np.cross(B - A, C - A)
    nn = np.einsum("ij,ij->i", nrm, nrm)
    h = np.einsum("ij,ij->i", x[None, :] - A, nrm) / np.where(nn > 0, nn, 1.0)
    proj = x[None, :] - h[:, None] * nrm
    # barycentric coordinates from signed sub-areas
    la = np.einsum("ij,ij->i", np.cross(C - B, proj - B), nrm)
    lb = np.einsum("ij,ij->i", np.cross(A - C, proj - C), nrm)
    lc = np.einsum("ij,ij->i", np.cross(B - A, proj - A), nrm)
    inside = (la >= 0) & (lb >= 0) & (lc >= 0) & (nn > 0)
    best = proj.copy()
    out = ~inside
    if out.any():
        X = np.broadcast_to(x, (int(out.sum()), 3))
        cands = [_segment_nearest(A[out], B[out], X), _segment_nearest(B[out], C[out], X),
                 _segment_nearest(C[out], A[out], X)]
        d = np.stack([np.einsum("ij,ij->i", q - X, q - X) for q in cands], axis=1)
        k = np.argmin(d, axis=1)
        best[out] = np.stack(cands, axis=1)[np.arange(len(k)), k]
    return best


def shrink(tris, own, p, n, r0, max_iter=100):
    """Shrinking ball tangent at p (inward normal n) against triangles
    `tris` except index `own`: (centre, radius, iterations)."""
    keep = np.ones(len(tris), dtype=bool)
    if own is not None and own >= 0:
        keep[own] = False
    T = tris[keep]
    p = np.asarray(p, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    r = float(r0)
    it = 0
    for it in range(max_iter):
        c = p + r * n
        q = nearest_points(T, c)
        d2 = np.einsum("ij,ij->i", q - c, q - c)
        k = int(np.argmin(d2))
        if np.sqrt(d2[k]) >= r * (1.0 - 1e-12):
            break
        pq = q[k] - p
        dn = float(pq @ n)
        rn = float(pq @ pq) / (2.0 * dn) if dn > 0 else np.inf
        if not (rn < r):
            break
        r = rn
    return p + r * n, r, it + 1


def boundary_triangles(w):
    """Boundary faces of a workload's tet mesh (faces in one tet only) as
    world-coordinate triangles (m, 3, 3) and their ids 4 * tet + face."""
    q, _, _ = w.ints()
    s = 1.0 / float(1 << w.grid_bits)
    T = w.tets.astype(np.int64)
    faces = {}
    opp = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))
    for t in range(len(T)):
        for f in range(4):
            key = tuple(sorted(int(T[t, c]) for c in opp[f]))
            faces.setdefault(key, []).append(4 * t + f)
    ids = sorted(v[0] for v in faces.values() if len(v) == 1)
    tris = np.array([[q[T[i >> 2, c]] * s for c in opp[i & 3]] for i in ids], dtype=np.float64).reshape(-1, 3, 3)
    return tris, np.array(ids, dtype=np.int64)
