"""Exact rational oracle for tiny inputs (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import anything under ``oracle/``; the library never does.

What it computes, written from the paper:

* Power distance  pd(x, m_i) = |x - theta_i|^2 - r_i^2  (Sec. 3.2, after Eq. 1).
* Power cell of m_i: points no farther (in power distance) from m_i than from
  any other sphere (Eq. 1); restricted cell RPC_i = cell cap shape (Eq. 2-3).
* Tet-Cell strategy (Sec. 5.2): the shape is a simplicial mesh; for every
  (simplex t, sphere i) pair the piece P(t,i) = t cap cell_i is obtained by
  clipping t successively with the half-spaces {pd(x,i) <= pd(x,k)} of the
  radical hyperplanes (Sec. 4.1.2).  This oracle clips against ALL other
  spheres by brute force, with exact rationals, so there is no neighbour
  search to get wrong.
* Restricted elements (Sec. 3.2 list): RPC_i, RPF_ij = RPC_i cap RPC_j,
  RPE_ijk, RPV_ijkl.  Inside one piece the element for {i} u J is the face of
  P(t,i) lying on the radical planes of J.
* Fractional Euler characteristic (Sec. 4.1.2, Eq. 7): every face of a piece
  is weighted by 1/n, n = number of mesh simplices sharing the lowest-
  dimensional mesh face that carries it (the paper's 1/2 for a vertex or edge
  shared by two triangles; new vertices inherit from the clipped edge, new
  edges from the clipped face, faces of the radical planes are interior and
  count 1).  chi(element) = sum over its faces of (-1)^dim * weight; the
  per-element counting formula V - E + F - C is from Sec. 4.1.
* Connected components (Sec. 4.1.1, "simple traversal"): pieces of one element
  in face-adjacent simplices are linked when the element crosses the shared
  facet; beta_0 = number of BFS components.
* Contractible iff beta_0 == 1 and chi == 1 (Sec. 3.3, Eq. 5-6; Sec. 4.1).

Generic position is assumed: a point exactly on a radical plane raises
``Degenerate`` (the library reports the same case as an error).
"""
from __future__ import annotations

from collections import defaultdict, deque
from fractions import Fraction
from itertools import combinations
from math import factorial


class Degenerate(Exception):
    pass


def power_distance(x, c, w):
    """pd(x, m) = |x - c|^2 - w with w = r^2 (Sec. 3.2)."""
    return sum((xi - ci) ** 2 for xi, ci in zip(x, c)) - w


def radical_halfspace(ci, wi, ck, wk):
    """Affine h with h(x) = pd(x, i) - pd(x, k); the cell of i keeps h <= 0."""
    a = tuple(2 * (b - a_) for a_, b in zip(ci, ck))
    b0 = (sum(v * v for v in ci) - wi) - (sum(v * v for v in ck) - wk)
    return a, b0


def _clip(verts, pid, a, b0, d):
    """Intersect a simple polytope (vertices with their plane incidences) with
    {a.x + b0 <= 0}.  Returns the new vertex list (empty if nothing is left)."""
    vals = [sum(ai * xi for ai, xi in zip(a, x)) + b0 for x, _ in verts]
    if any(v == 0 for v in vals):
        raise Degenerate("vertex on a radical plane")
    ins = [n for n, v in enumerate(vals) if v < 0]
    outs = [n for n, v in enumerate(vals) if v > 0]
    if not outs:
        return verts
    if not ins:
        return []
    new = []
    for i in ins:
        xi, inci = verts[i]
        for o in outs:
            xo, inco = verts[o]
            common = inci & inco
            if len(common) == d - 1:          # i, o are the two ends of an edge
                lam = Fraction(vals[i]) / (vals[i] - vals[o])
                x = tuple(p + lam * (q - p) for p, q in zip(xi, xo))
                new.append((x, common | {pid}))
    return [verts[i] for i in ins] + new


def _faces(verts):
    """All faces of a simple polytope as plane sets (frozensets); the empty set
    is the polytope itself."""
    fs = set()
    for _, inc in verts:
        for m in range(len(inc) + 1):
            for q in combinations(sorted(inc), m):
                fs.add(frozenset(q))
    return fs


def _triangulate(verts, Q, d):
    """Pulling triangulation of face Q: list of vertex-index simplices."""
    vs = [n for n, (_, inc) in enumerate(verts) if Q <= inc]
    if len(Q) == d:
        return [[vs[0]]]
    apex = vs[0]
    planes = set().union(*[verts[n][1] for n in vs]) - Q
    out = []
    for p in sorted(planes):
        if p in verts[apex][1]:
            continue
        Q2 = Q | {p}
        if not any(Q2 <= verts[n][1] for n in vs):
            continue
        for s in _triangulate(verts, Q2, d):
            out.append([apex] + s)
    return out


def _det(rows):
    n = len(rows)
    if n == 1:
        return rows[0][0]
    if n == 2:
        return rows[0][0] * rows[1][1] - rows[0][1] * rows[1][0]
    tot = 0
    for c in range(n):
        minor = [r[:c] + r[c + 1:] for r in rows[1:]]
        tot += (-1) ** c * rows[0][c] * _det(minor)
    return tot


def volume_and_moment(verts, d):
    """Exact volume and first moment (integral of x) of a convex polytope."""
    vol = Fraction(0)
    mom = [Fraction(0)] * d
    for s in _triangulate(verts, frozenset(), d):
        x0 = verts[s[0]][0]
        rows = [[verts[n][0][k] - x0[k] for k in range(d)] for n in s[1:]]
        v = abs(Fraction(_det(rows))) / factorial(d)
        vol += v
        for k in range(d):
            mom[k] += v * sum(Fraction(verts[n][0][k]) for n in s) / (d + 1)
    return vol, mom


def rpd_exact(points, simplices, centers, weights, mutate=None):
    """Brute-force restricted power diagram of a simplicial mesh (any dimension).

    points   : list of integer coordinate tuples (the mesh vertices)
    simplices: list of (d+1)-tuples of point indices, positively oriented
    centers  : list of integer coordinate tuples, weights: list of ints (= r^2)

    Returns a dict with
      'pieces'  : {(t, i): (volume, moment)} for every nonempty piece
      'chi'     : {key: Fraction} fractional Euler characteristic (1/n weights)
      'chi_own' : {key: int} the same with each shared mesh face given to its
                  lowest-numbered simplex (the library's integer form)
      'beta0'   : {key: int} connected components
      'flag'    : {key: bool} contractible (beta0 == 1 and chi == 1)
      'chi_piece': {(t, key): Fraction} the contribution of simplex t
      'chi_plain': {(t, i): int} unweighted V - E + F - C of each piece
      'wcount'  : {(t, i): [w_0, ..., w_d]} weighted number of faces of each
                  dimension of the piece (w_d counts the piece itself)
    Keys are sorted sphere-index tuples of length 1 (RPC), 2 (RPF), 3 (RPE),
    4 (RPV, in 3D).

    ``mutate`` plants a known mistake so the tests can show that the pins
    catch it: "unit_weights" (no fractional sharing), "drop_cell" (no -C term),
    "wrong_side" (keep the far side of each radical plane), "skip_last" (never
    clip against the last sphere).
    """
    d = len(points[0])
    S = len(simplices)
    ns = len(centers)
    # mesh faces -> simplices containing them (for the 1/n weights and owners)
    star = defaultdict(list)
    for t, simp in enumerate(simplices):
        for m in range(1, d + 1):
            for f in combinations(sorted(simp), m):
                star[frozenset(f)].append(t)
    # facet adjacency
    facet_of = defaultdict(list)
    for t, simp in enumerate(simplices):
        for f in range(d + 1):
            facet_of[frozenset(simp[:f] + simp[f + 1:])].append((t, f))
    adj = [[-1] * (d + 1) for _ in range(S)]
    for lst in facet_of.values():
        if len(lst) == 2:
            (t1, f1), (t2, f2) = lst
            adj[t1][f1] = t2
            adj[t2][f2] = t1
    cw = [(tuple(c), w) for c, w in zip(centers, weights)]

    pieces = {}
    chi = defaultdict(Fraction)
    chi_own = defaultdict(int)
    chi_piece = {}
    chi_plain = {}
    wcount = {}
    nodes = defaultdict(dict)   # key -> {t: [facets linked]}
    for t, simp in enumerate(simplices):
        P = [tuple(points[v]) for v in simp]
        cen = tuple(Fraction(sum(p[k] for p in P), d + 1) for k in range(d))
        order = sorted(range(ns), key=lambda k: power_distance(cen, *cw[k]))
        for i in range(ns):
            verts = [(P[a], frozenset(f for f in range(d + 1) if f != a)) for a in range(d + 1)]
            for k in order:
                if k == i or (mutate == "skip_last" and k == ns - 1):
                    continue
                a, b0 = radical_halfspace(cw[i][0], cw[i][1], cw[k][0], cw[k][1])
                if mutate == "wrong_side":
                    a, b0 = tuple(-v for v in a), -b0
                verts = _clip(verts, d + 1 + k, a, b0, d)
                if not verts:
                    break
            if len(verts) < d + 1:
                continue
            pieces[(t, i)] = volume_and_moment(verts, d)
            faces = _faces(verts)
            chi_plain[(t, i)] = sum((-1) ** (d - len(Q)) for Q in faces)
            wdim = [Fraction(0)] * (d + 1)

            def carrier(Q):
                fac = [f for f in Q if f <= d]
                if not fac:
                    return None
                return frozenset(simp[c] for c in range(d + 1) if c not in fac)

            weight = {}
            own = {}
            for Q in faces:
                car = carrier(Q)
                if car is None:
                    weight[Q], own[Q] = Fraction(1), 1
                    if mutate == "drop_cell" and not Q:
                        weight[Q], own[Q] = Fraction(0), 0
                elif mutate == "unit_weights":
                    weight[Q], own[Q] = Fraction(1), 1
                else:
                    sh = star[car]
                    weight[Q] = Fraction(1, len(sh))
                    own[Q] = 1 if t == min(sh) else 0
                wdim[d - len(Q)] += weight[Q]
            wcount[(t, i)] = wdim
            bis = sorted({p for Q in faces for p in Q if p > d})
            for m in range(0, d + 1):
                for J in combinations(bis, m):
                    J = frozenset(J)
                    if J not in faces:
                        continue
                    ks = sorted(p - d - 1 for p in J)
                    if ks and ks[0] < i:
                        continue     # emitted by the lowest sphere of the key
                    key = tuple([i] + ks)
                    sub = [Q for Q in faces if J <= Q]
                    c_frac = sum((-1) ** (d - len(Q)) * weight[Q] for Q in sub)
                    chi_piece[(t, key)] = c_frac
                    chi[key] += c_frac
                    chi_own[key] += sum((-1) ** (d - len(Q)) * own[Q] for Q in sub)
                    links = [f for f in range(d + 1) if adj[t][f] >= 0 and (J | {f}) in faces]
                    nodes[key][t] = links

    beta0 = {}
    for key, nd in nodes.items():
        seen = set()
        comp = 0
        for t0 in nd:
            if t0 in seen:
                continue
            comp += 1
            dq = deque([t0])
            seen.add(t0)
            while dq:
                t = dq.popleft()
                for f in nd[t]:
                    t2 = adj[t][f]
                    if t2 not in nd:
                        raise AssertionError(f"link target missing for {key}: {t}->{t2}")
                    if t2 not in seen:
                        seen.add(t2)
                        dq.append(t2)
        beta0[key] = comp
    flag = {k: (beta0[k] == 1 and chi[k] == 1) for k in beta0}
    return {'pieces': pieces, 'chi': dict(chi), 'chi_own': dict(chi_own), 'beta0': beta0, 'flag': flag,
            'adj': adj, 'chi_piece': chi_piece, 'chi_plain': chi_plain, 'wcount': wcount}


def mesh_euler(simplices):
    """chi of a simplicial complex = sum over its faces of (-1)^dim (Sec. 6)."""
    fs = set()
    for simp in simplices:
        for m in range(1, len(simp) + 1):
            for f in combinations(sorted(simp), m):
                fs.add(f)
    return sum((-1) ** (len(f) - 1) for f in fs)


def from_workload(w):
    """Integer inputs of a seeded workload for ``rpd_exact``."""
    q, c, r = w.ints()
    pts = [tuple(int(v) for v in row) for row in q]
    simp = [tuple(int(v) for v in row) for row in w.tets]
    cen = [tuple(int(v) for v in row) for row in c]
    wts = [int(v) * int(v) for v in r]
    return pts, simp, cen, wts
