"""Medial mesh thinning on the CPU (TEST INFRASTRUCTURE ONLY: only tests/ use it).

Sec. 5.3, restated plainly: the complex has edges, triangles and tetrahedra
given by sorted sphere-index keys.  A simple pair (x, y) is a simplex x with
a face y that no other simplex of the complex has as a face.  Every triangle
f has an importance alpha(f) = |RPE_f| / mean of the three spheres'
diameters.  Step 1: while a tetrahedron remains, remove the tet-triangle
simple pair whose triangle has the smallest importance.  Step 2: while some
triangle that was a face of an original tetrahedron (and is now the face of
no tetrahedron) has an edge that no other triangle contains, and its
importance is below sigma, remove the one with the smallest importance
together with that edge.  Ties: the smaller triangle key; a triangle with
several free edges gives up the edge with the smallest key (readings of the
paper, which does not fix them).

Plain loops that rescan everything at each removal; no code is shared with
the library.
"""
from __future__ import annotations

from itertools import combinations


def thin(edges, faces, alpha, tets, sigma):
    """edges/faces/tets: lists of sorted key tuples; alpha: {face: importance}.
    Returns (edges, faces, tets) left after thinning, each sorted."""
    E = set(map(tuple, edges))
    F = set(map(tuple, faces))
    T = set(map(tuple, tets))
    orig = {f for t in T for f in combinations(t, 3)}

    def tets_of(f):
        return [t for t in T if set(f) <= set(t)]

    def faces_of(e):
        return [f for f in F if set(e) <= set(f)]

    while T:
        cands = [f for f in F if len(tets_of(f)) == 1]
        if not cands:
            break
        f = min(cands, key=lambda x: (alpha[x], x))
        T.discard(tets_of(f)[0])
        F.discard(f)
    while True:
        best = None
        for f in sorted(F):
            if f not in orig or tets_of(f) or not (alpha[f] < sigma):
                continue
            free = [e for e in combinations(f, 2) if e in E and len(faces_of(e)) == 1]
            if free and (best is None or (alpha[f], f) < (alpha[best[0]], best[0])):
                best = (f, min(free))
        if best is None:
            break
        F.discard(best[0])
        E.discard(best[1])
    return sorted(E), sorted(F), sorted(T)
