"""Seeded tetrahedral meshes from a jittered lattice (input generator only).

A shape is given by a signed distance function (negative inside).  The
generator lays a lattice of spacing ``h`` over the shape's bounding box,
jitters the lattice points, snaps them to the integer grid of spacing
``2**-grid_bits``, splits every lattice cube into the six Freudenthal (Kuhn)
tetrahedra that share the cube's main diagonal, keeps the tetrahedra whose
centroid lies inside the shape, and then removes tetrahedra until the kept
set is a manifold solid with one face-connected component.

The paper assumes its input is a manifold tetrahedral mesh with one connected
component and no cavity (Sec. 3.3, Assumption); ``validate`` reports those
properties so that callers can reject a seed that violates them.

This module computes mesh topology and geometry for building inputs; it holds
none of the restricted-power-diagram arithmetic.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

# Cube corner c = x + 2y + 4z; each tet walks 0 -> e_a -> e_a+e_b -> 7.
KUHN = np.array([(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7),
                 (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)], dtype=np.int64)
# Face f of a tet is the triangle opposite local vertex f.
FACE_LOCAL = np.array([(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)], dtype=np.int64)
EDGE_LOCAL = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], dtype=np.int64)

MAX_COORD = (1 << 21) - 1   # |integer coordinate| bound assumed by the library


def snap(x: np.ndarray, grid_bits: int) -> np.ndarray:
    """Round to the grid 2**-grid_bits (round half to even, like rint)."""
    return np.rint(np.asarray(x, dtype=np.float64) * float(1 << grid_bits)).astype(np.int64)


def orient_int(q: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Exact sign of det[p1-p0, p2-p0, p3-p0] for integer points (local coords)."""
    p0 = q[tets[:, 0]]
    a = q[tets[:, 1]] - p0
    b = q[tets[:, 2]] - p0
    c = q[tets[:, 3]] - p0
    if max(np.abs(a).max(initial=0), np.abs(b).max(initial=0), np.abs(c).max(initial=0)) >= (1 << 20):
        # fall back to Python integers for long edges
        out = np.empty(len(tets), dtype=np.int64)
        for n in range(len(tets)):
            ax, ay, az = (int(v) for v in a[n])
            bx, by, bz = (int(v) for v in b[n])
            cx, cy, cz = (int(v) for v in c[n])
            d = ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx)
            out[n] = (d > 0) - (d < 0)
        return out
    cr = np.cross(b, c)              # |.| < 2^41
    d = np.einsum('ij,ij->i', a, cr)  # |.| < 3 * 2^61
    return np.sign(d)


def _unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (what np.unique returns), by a sort: much faster
    than the hashing np.unique on the multi-million-key arrays used here."""
    s = np.sort(np.asarray(x).ravel())
    if s.size == 0:
        return s
    keep = np.empty(s.size, dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def _face_keys(tets: np.ndarray, nv: int) -> np.ndarray:
    f = np.sort(tets[:, FACE_LOCAL], axis=2)          # (T,4,3)
    return (f[..., 0] * nv + f[..., 1]) * nv + f[..., 2]


def _edge_keys(tets: np.ndarray, nv: int) -> np.ndarray:
    e = np.sort(tets[:, EDGE_LOCAL], axis=2)          # (T,6,2)
    return e[..., 0] * nv + e[..., 1]


def face_adjacency(tets: np.ndarray, nv: int):
    """adj[t,f] = tet across face f (-1 on the boundary); also the face counts."""
    T = len(tets)
    keys = _face_keys(tets, nv).ravel()
    order = np.argsort(keys, kind='stable')
    sk = keys[order]
    head = np.empty(sk.size, dtype=bool)
    if sk.size:
        head[0] = True
        np.not_equal(sk[1:], sk[:-1], out=head[1:])
    start = np.nonzero(head)[0]
    counts = np.diff(np.append(start, sk.size))
    if counts.size and counts.max() > 2:
        raise ValueError("a face is shared by more than two tets")
    adj = -np.ones(4 * T, dtype=np.int64)
    pairs = start[counts == 2]
    a = order[pairs]
    b = order[pairs + 1]
    adj[a] = b // 4
    adj[b] = a // 4
    return adj.reshape(T, 4), counts


def _vertex_badness(tets: np.ndarray, nv: int):
    """Per vertex: number of face-connected tet clusters around it and the Euler
    characteristic of its link (a disk has 1, a sphere 2)."""
    T = len(tets)
    adj, fcounts = face_adjacency(tets, nv)
    # graph on (tet, local vertex) corners, joined through interior faces
    t_idx, f_idx = np.nonzero(adj > np.arange(T)[:, None])
    t2 = adj[t_idx, f_idx]
    rows, cols = [], []
    for k in range(3):
        lv = FACE_LOCAL[f_idx, k]
        gv = tets[t_idx, lv]
        # local index of gv inside t2
        l2 = np.argmax(tets[t2] == gv[:, None], axis=1)
        rows.append(4 * t_idx + lv)
        cols.append(4 * t2 + l2)
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    g = coo_matrix((np.ones(len(rows), dtype=np.int8), (rows, cols)), shape=(4 * T, 4 * T))
    _, lab = connected_components(g, directed=False)
    corner_v = tets.ravel()
    pair = _unique(corner_v.astype(np.int64) * (4 * T) + lab)
    clusters = np.bincount(pair // (4 * T), minlength=nv)
    # link Euler characteristic: (#edges at v) - (#faces at v) + (#tets at v)
    ek = _unique(_edge_keys(tets, nv))
    nedge = np.bincount(ek // nv, minlength=nv) + np.bincount(ek % nv, minlength=nv)
    fk = _unique(_face_keys(tets, nv))
    fa, fb, fc = fk // (nv * nv), (fk // nv) % nv, fk % nv
    nface = np.bincount(fa, minlength=nv) + np.bincount(fb, minlength=nv) + np.bincount(fc, minlength=nv)
    ntet = np.bincount(corner_v, minlength=nv)
    chi_link = nedge - nface + ntet
    return clusters, chi_link, lab


def _largest_component(tets: np.ndarray, nv: int) -> np.ndarray:
    T = len(tets)
    adj, _ = face_adjacency(tets, nv)
    t_idx, f_idx = np.nonzero(adj >= 0)
    g = coo_matrix((np.ones(len(t_idx), dtype=np.int8), (t_idx, adj[t_idx, f_idx])), shape=(T, T))
    n, lab = connected_components(g, directed=False)
    if n <= 1:
        return tets
    big = np.argmax(np.bincount(lab))
    return tets[lab == big]


def make_manifold(tets: np.ndarray, nv: int, max_iter: int = 64) -> np.ndarray:
    """Remove tets until every vertex star is a single face-connected cluster
    whose link is a disk or a sphere (which also makes every edge manifold)."""
    for _ in range(max_iter):
        tets = _largest_component(tets, nv)
        clusters, chi_link, lab = _vertex_badness(tets, nv)
        used = np.bincount(tets.ravel(), minlength=nv) > 0
        bad = used & ((clusters != 1) | ((chi_link != 1) & (chi_link != 2)))
        if not bad.any():
            return tets
        T = len(tets)
        drop = np.zeros(T, dtype=bool)
        corner_v = tets.ravel()
        corner_bad = bad[corner_v]
        # keep only the biggest cluster around a multi-cluster vertex
        cb = np.nonzero(corner_bad)[0]
        v_of = corner_v[cb]
        l_of = lab[cb]
        key = v_of.astype(np.int64) * (4 * T) + l_of
        uk, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
        best = {}
        for k_, c_ in zip(uk, cnt):
            v_ = int(k_ // (4 * T))
            if v_ not in best or c_ > best[v_][1]:
                best[v_] = (int(k_), int(c_))
        for n_, c in enumerate(cb):
            v_ = int(v_of[n_])
            single = clusters[v_] == 1
            if single or key[n_] != best[v_][0]:
                drop[c // 4] = True
        tets = tets[~drop]
    raise RuntimeError("mesh cleaning did not converge")


def compact(q: np.ndarray, tets: np.ndarray):
    used = _unique(tets)
    remap = -np.ones(len(q), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return q[used], remap[tets]


def validate(q: np.ndarray, tets: np.ndarray) -> dict:
    """Orientation, manifoldness, components, boundary shells and chi of a mesh."""
    nv, T = len(q), len(tets)
    info = {}
    info['orient_min'] = int(orient_int(q, tets).min()) if T else 0
    adj, fcounts = face_adjacency(tets, nv)
    clusters, chi_link, _ = _vertex_badness(tets, nv)
    used = np.bincount(tets.ravel(), minlength=nv) > 0
    info['manifold'] = bool(np.all(~used | ((clusters == 1) & ((chi_link == 1) | (chi_link == 2)))))
    t_idx, f_idx = np.nonzero(adj >= 0)
    g = coo_matrix((np.ones(len(t_idx), dtype=np.int8), (t_idx, adj[t_idx, f_idx])), shape=(T, T))
    info['components'] = int(connected_components(g, directed=False)[0])
    # boundary shells: boundary faces joined through shared edges
    bt, bf = np.nonzero(adj < 0)
    nb = len(bt)
    if nb:
        tri = np.sort(tets[bt[:, None], FACE_LOCAL[bf]], axis=1)
        ek = np.concatenate([tri[:, 0] * nv + tri[:, 1], tri[:, 0] * nv + tri[:, 2], tri[:, 1] * nv + tri[:, 2]])
        fid = np.concatenate([np.arange(nb)] * 3)
        o = np.argsort(ek, kind='stable')
        ek, fid = ek[o], fid[o]
        same = ek[1:] == ek[:-1]
        gb = coo_matrix((np.ones(int(same.sum()), np.int8), (fid[:-1][same], fid[1:][same])), shape=(nb, nb))
        info['shells'] = int(connected_components(gb, directed=False)[0])
    else:
        info['shells'] = 0
    nE = len(_unique(_edge_keys(tets, nv)))
    nF = len(_unique(_face_keys(tets, nv)))
    info['V'], info['E'], info['F'], info['T'] = int(used.sum()), int(nE), int(nF), int(T)
    info['chi'] = int(used.sum()) - nE + nF - T
    return info


def project_boundary(q, tets, sdf, grid_bits: int, min_ratio: float = 0.02, rounds: int = 12):
    """Move the boundary vertices of a carved lattice mesh onto the surface
    {sdf = 0}: one Newton step x - sdf(x) grad(sdf)(x) (exact for planes and
    cylinders), on the integer grid.  A vertex whose move would leave one of
    its tets with less than `min_ratio` of its volume (or inverted) has the
    move halved, round after round; whatever is still too flat keeps its
    original position.  Topology is unchanged.  Returns new coordinates."""
    scale = 1.0 / float(1 << grid_bits)
    faces = np.sort(np.concatenate([tets[:, list(f)] for f in FACE_LOCAL], axis=0), axis=1)
    uf, cnt = np.unique(faces, axis=0, return_counts=True)
    bv = np.unique(uf[cnt == 1].ravel())
    x = q[bv].astype(np.float64) * scale
    f = sdf(x)
    eps = 1e-6 * max(1.0, float(np.abs(x).max()))
    grad = np.stack([(sdf(x + eps * e) - sdf(x - eps * e)) / (2 * eps) for e in np.eye(3)], axis=1)
    grad /= np.maximum(np.linalg.norm(grad, axis=1, keepdims=True), 1e-12)
    disp = -f[:, None] * grad
    on_b = np.zeros(len(q), dtype=bool)
    on_b[bv] = True
    tb = tets[on_b[tets].any(axis=1)]
    pos = np.full(len(q), -1, dtype=np.int64)
    pos[bv] = np.arange(len(bv))

    def volumes(qq):
        p0 = qq[tb[:, 0]].astype(np.float64)
        return np.einsum("ij,ij->i", qq[tb[:, 1]] - p0, np.cross(qq[tb[:, 2]] - p0, qq[tb[:, 3]] - p0))

    v0 = volumes(q)
    fac = np.ones(len(bv))
    qn = q
    for it in range(rounds + 64):
        qn = q.copy()
        qn[bv] = snap(x + fac[:, None] * disp, grid_bits)
        bad = ~(volumes(qn) > min_ratio * v0)
        if not bad.any():
            break
        vb = np.unique(tb[bad].ravel())
        vb = vb[on_b[vb]]
        # halve the moves of the vertices of too-flat tets; after `rounds`
        # halvings they stay where the carving put them
        fac[pos[vb]] = fac[pos[vb]] * 0.5 if it < rounds else 0.0
    if np.any(orient_int(qn, tets) <= 0):   # exact check; fall back to the carved mesh
        return q
    return qn


def lattice_mesh(sdf, lo, hi, h: float, grid_bits: int, rng: np.random.Generator,
                 jitter: float = 0.1, inside_by_vertices: bool = False, project: bool = False):
    """Jittered Freudenthal lattice restricted to {sdf < 0}, cleaned to a manifold.

    Returns (integer vertex coordinates int64[nv,3], tets int64[nt,4]) with every
    tet positively oriented.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = np.maximum(np.ceil((hi - lo) / h).astype(np.int64), 1)
    nx, ny, nz = (int(v) for v in n)
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing='ij')
    idx = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], axis=1)
    p = lo + h * idx + rng.uniform(-jitter * h, jitter * h, size=idx.shape)
    q = snap(p, grid_bits)
    if np.abs(q).max() > MAX_COORD:
        raise ValueError("coordinates exceed the integer grid bound; lower grid_bits")
    vid = lambda i, j, k: (i * (ny + 1) + j) * (nz + 1) + k
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing='ij')
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    corners = np.stack([vid(ci + (c & 1), cj + ((c >> 1) & 1), ck + ((c >> 2) & 1)) for c in range(8)], axis=1)
    scale = 1.0 / float(1 << grid_bits)
    if inside_by_vertices:
        sv = sdf(q * scale)
    keep_t = []
    chunk = 1 << 18
    for s in range(0, len(corners), chunk):
        cc = corners[s:s + chunk]
        tt = cc[:, KUHN].reshape(-1, 4)
        if inside_by_vertices:
            inside = sv[tt].mean(axis=1) < 0
        else:
            cen = q[tt].mean(axis=1) * scale
            inside = sdf(cen) < 0
        keep_t.append(tt[inside])
    tets = np.concatenate(keep_t, axis=0)
    o = orient_int(q, tets)
    if np.any(o == 0):
        raise ValueError("flat tetrahedron after jitter")
    neg = o < 0
    tets[neg] = tets[neg][:, [0, 1, 3, 2]]
    tets = make_manifold(tets, len(q))
    q, tets = compact(q, tets)
    if project:
        q = project_boundary(q, tets, sdf, grid_bits)
    return q, tets


def slab_mesh(half, holes, hole_r: float, h: float, grid_bits: int, rng: np.random.Generator,
              jitter: float = 0.1, min_ratio: float = 0.02, rounds: int = 12):
    """Tet mesh of the box [-half, half] with z-through cylindrical holes of
    radius hole_r centred at (x, 0) for x in `holes`, with an exactly planar
    box boundary, as a surface-fitting tetrahedralisation gives.

    The lattice spacing is the largest h' <= h that divides every side; whole
    lattice cubes (six Kuhn tets each) are kept when their centre lies outside
    every hole.  Vertices move by up to `jitter` h' along each axis except the
    axes of the box planes they lie on, so the box faces stay flat.  The
    corners of removed cubes (the hole walls) are then moved radially in x-y
    onto the nearest cylinder, z kept; a move that would leave a tet with less
    than `min_ratio` of its volume is halved, round after round, and after
    `rounds` halvings dropped.  Returns integer coordinates and tets."""
    half = np.asarray(half, dtype=np.float64)
    m = int(np.ceil(1.0 / h - 1e-9))
    while np.any(np.abs(2 * half * m - np.round(2 * half * m)) > 1e-9):
        m += 1
    hh = 1.0 / m
    n = np.round(2 * half * m).astype(np.int64)
    nx, ny, nz = (int(v) for v in n)
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing='ij')
    idx = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], axis=1)
    on_plane = (idx == 0) | (idx == n[None, :])
    jit = rng.uniform(-jitter * hh, jitter * hh, size=idx.shape)
    jit[on_plane] = 0.0
    p = -half + hh * idx + jit
    vid = lambda i, j, k: (i * (ny + 1) + j) * (nz + 1) + k
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing='ij')
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    cen = -half + hh * (np.stack([ci, cj, ck], axis=1) + 0.5)
    keep = np.ones(len(ci), dtype=bool)
    for cx in holes:
        keep &= np.hypot(cen[:, 0] - cx, cen[:, 1]) >= hole_r
    corners = np.stack([vid(ci + (c & 1), cj + ((c >> 1) & 1), ck + ((c >> 2) & 1)) for c in range(8)], axis=1)
    wall = np.zeros(len(p), dtype=bool)
    wall[np.unique(corners[~keep].ravel())] = True
    tets = corners[keep][:, KUHN].reshape(-1, 4)
    q = snap(p, grid_bits)
    if np.abs(q).max() > MAX_COORD:
        raise ValueError("coordinates exceed the integer grid bound; lower grid_bits")
    o = orient_int(q, tets)
    if np.any(o == 0):
        raise ValueError("flat tetrahedron after jitter")
    neg = o < 0
    tets[neg] = tets[neg][:, [0, 1, 3, 2]]
    tets = make_manifold(tets, len(q))
    used = np.zeros(len(q), dtype=bool)
    used[tets.ravel()] = True
    wv = np.where(wall & used)[0]
    if len(holes) and len(wv):
        hc = np.asarray(holes, dtype=np.float64)
        x = p[wv]
        k = np.argmin(np.abs(np.hypot(x[:, None, 0] - hc[None, :], x[:, None, 1]) - hole_r), axis=1)
        dx, dy = x[:, 0] - hc[k], x[:, 1]
        rad = np.maximum(np.hypot(dx, dy), 1e-12)
        disp = np.zeros_like(x)
        disp[:, 0] = dx * (hole_r / rad - 1.0)
        disp[:, 1] = dy * (hole_r / rad - 1.0)
        disp[on_plane[wv]] = 0.0   # a wall vertex on an x or y box plane keeps that coordinate
        on_w = np.zeros(len(q), dtype=bool)
        on_w[wv] = True
        tb = tets[on_w[tets].any(axis=1)]
        pos = np.full(len(q), -1, dtype=np.int64)
        pos[wv] = np.arange(len(wv))

        def volumes(qq):
            p0 = qq[tb[:, 0]].astype(np.float64)
            return np.einsum("ij,ij->i", qq[tb[:, 1]] - p0, np.cross(qq[tb[:, 2]] - p0, qq[tb[:, 3]] - p0))

        v0 = volumes(q)
        fac = np.ones(len(wv))
        qn = q
        for it in range(rounds + 64):
            qn = q.copy()
            qn[wv] = snap(x + fac[:, None] * disp, grid_bits)
            bad = ~(volumes(qn) > min_ratio * v0)
            if not bad.any():
                break
            vb = np.unique(tb[bad].ravel())
            vb = vb[on_w[vb]]
            fac[pos[vb]] = fac[pos[vb]] * 0.5 if it < rounds else 0.0
        if not np.any(orient_int(qn, tets) <= 0):
            q = qn
    return compact(q, tets)
