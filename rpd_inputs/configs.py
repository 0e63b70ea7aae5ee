"""Named seeded workloads (input generator only).

* ``torus_c1``  solid torus R=1, r=0.4, ~5k tets, 64 core-circle spheres, k=16
* ``block_c2``  4x2x1 box with three z-through holes (genus 3), ~200k tets,
  2k near-medial spheres, k=32
* ``blob_c3``   union of 200 ellipsoids, ~2M tets, 20k near-medial spheres
* ``tiny_*``    <= 48 tets (box, 2x2x1 block, ring torus) with 1-12 spheres

The paper measures on ABC CAD models and organic models (Sec. 6), which are not
available here; these synthetic shapes stand in for them with the paper's mesh
and sphere counts (#t 1k-10k, #s up to ~12k; Table 4 and Fig. 14).

All coordinates and radii are exact multiples of 2**-grid_bits, so snapping to
the library's integer grid is the identity on them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mesh import lattice_mesh, slab_mesh, validate, snap, MAX_COORD, orient_int, KUHN, compact
from .shapes import (torus_sdf, torus_core_spheres, block_sdf, block_medial_spheres,
                     BLOCK_HALF, EllipsoidBlob, slab_holes, slab_sdf, slab_medial_spheres)

BASE_SEED = 20240318


@dataclass
class Workload:
    name: str
    verts: np.ndarray      # float64 [nv,3], multiples of 2**-grid_bits
    tets: np.ndarray       # int32 [nt,4], positively oriented
    centers: np.ndarray    # float64 [ns,3]
    radii: np.ndarray      # float64 [ns]
    grid_bits: int
    k: int = 16
    precision: str = "fp64"
    info: dict = field(default_factory=dict)

    @property
    def nt(self):
        return len(self.tets)

    @property
    def ns(self):
        return len(self.radii)

    def ints(self):
        """Integer grid coordinates (int64) of vertices, centres and radii."""
        return (snap(self.verts, self.grid_bits), snap(self.centers, self.grid_bits),
                snap(self.radii, self.grid_bits))


def _snap_spheres(c, r, g):
    ci = snap(c, g)
    ri = np.maximum(snap(r, g), 0)
    key = np.concatenate([ci, ri[:, None]], axis=1)
    _, first = np.unique(key, axis=0, return_index=True)
    first = np.sort(first)
    s = 1.0 / float(1 << g)
    return ci[first] * s, ri[first] * s


def _grid_bits_for(extent: float) -> int:
    g = 0
    while (extent * 1.05 + 0.1) * float(1 << (g + 1)) < MAX_COORD:
        g += 1
    return g


def _finish(name, q, tets, c, r, g, k, precision, expect_chi=None):
    info = validate(q, tets)
    if info['orient_min'] <= 0 or not info['manifold'] or info['components'] != 1 or info['shells'] != 1:
        raise ValueError(f"{name}: generated mesh violates the input assumption: {info}")
    if expect_chi is not None and info['chi'] != expect_chi:
        raise ValueError(f"{name}: chi {info['chi']} != {expect_chi}")
    s = 1.0 / float(1 << g)
    c, r = _snap_spheres(c, r, g)
    return Workload(name, q * s, tets.astype(np.int32), c, r, g, k, precision, info)


def torus_c1(seed: int = BASE_SEED, h: float = 0.155, ns: int = 64):
    rng = np.random.default_rng(seed)
    g = 20
    q, tets = lattice_mesh(torus_sdf(1.0, 0.4), [-1.45, -1.45, -0.45], [1.45, 1.45, 0.45], h, g, rng)
    c, r = torus_core_spheres(ns, rng)
    return _finish("torus_c1", q, tets, c, r, g, 16, "fp64", expect_chi=0)


def block_c2(seed: int = BASE_SEED + 1, h: float = 0.06, ns: int = 2000):
    rng = np.random.default_rng(seed)
    g = 19
    q, tets = lattice_mesh(block_sdf, -BLOCK_HALF - 0.01, BLOCK_HALF + 0.01, h, g, rng)
    c, r = block_medial_spheres(ns, rng)
    return _finish("block_c2", q, tets, c, r, g, 32, "fp32", expect_chi=-2)


def blob_c3(seed: int = BASE_SEED + 2, target_tets: int = 2_000_000, ns: int = 20000,
            n_ellipsoids: int = 200):
    rng = np.random.default_rng(seed)
    blob = EllipsoidBlob(n_ellipsoids, rng)
    # volume estimate -> lattice spacing for the target tet count
    p = rng.uniform(blob.lo, blob.hi, size=(200000, 3))
    frac = float((blob.sdf(p) < 0).mean())
    vol = frac * float(np.prod(blob.hi - blob.lo))
    h = (6.0 * vol / target_tets) ** (1.0 / 3.0)
    ext = float(np.abs(np.concatenate([blob.lo, blob.hi])).max()) + h
    g = _grid_bits_for(ext)
    q, tets = lattice_mesh(blob.sdf, blob.lo - h, blob.hi + h, h, g, rng, inside_by_vertices=True)
    c, r = blob.medial_spheres(ns, rng)
    return _finish("blob_c3", q, tets, c, r, g, 32, "fp32")


def genus_slab(genus: int, seed: int = BASE_SEED + 4, h: float = 0.075, ns: int = 256, hole_r: float = 0.2,
               project: bool = True):
    """A 4x2x1 slab with `genus` z-through holes (genus 0-5; chi = 1 - genus),
    ~100k tets at h = 0.075, and `ns` near-medial starting spheres: the
    topology-repair workload (many shapes of genus 0-5 from 256 spheres)."""
    rng = np.random.default_rng(seed + 97 * genus)
    g = 19
    holes = slab_holes(genus)
    if project:
        # flat box faces and hole walls on their cylinders, as a
        # surface-fitting tetrahedralisation places them
        q, tets = slab_mesh(BLOCK_HALF, holes, hole_r, h, g, rng)
    else:
        # a jittered lattice staircase (a rough, non-fitted boundary)
        q, tets = lattice_mesh(slab_sdf(holes, hole_r), -BLOCK_HALF - 0.01, BLOCK_HALF + 0.01, h, g, rng)
    c, r = slab_medial_spheres(ns, rng, holes, hole_r)
    w = _finish(f"genus{genus}_slab", q, tets, c, r, g, 32, "fp32", expect_chi=1 - genus)
    w.info["genus"] = genus
    return w


# ------------------------------------------------------------------ tiny set
def _cube_mesh(cells, h, g, rng, jitter_interior=0.0):
    """Union of lattice cubes (list of integer (i,j,k)), Kuhn-split."""
    cells = np.asarray(cells, dtype=np.int64)
    lo = cells.min(axis=0)
    hi = cells.max(axis=0) + 1
    dims = hi - lo + 1
    gi, gj, gk = np.meshgrid(*[np.arange(d) for d in dims], indexing='ij')
    idx = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], axis=1)
    p = (idx + lo) * h
    if jitter_interior > 0:
        interior = np.all((idx > 0) & (idx < dims - 1), axis=1)
        p[interior] += rng.uniform(-jitter_interior * h, jitter_interior * h, size=(int(interior.sum()), 3))
    q = snap(p, g)
    vid = lambda a: (a[:, 0] * dims[1] + a[:, 1]) * dims[2] + a[:, 2]
    rel = cells - lo
    corners = np.stack([vid(rel + np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])) for c in range(8)], axis=1)
    tets = corners[:, KUHN].reshape(-1, 4)
    o = orient_int(q, tets)
    tets[o < 0] = tets[o < 0][:, [0, 1, 3, 2]]
    return compact(q, tets)


TINY_SHAPES = {
    "box": [(i, j, k) for i in range(2) for j in range(2) for k in range(2)],       # 48 tets, convex
    "block": [(i, j, 0) for i in range(2) for j in range(2)],                         # 24 tets, convex
    "ring": [(i, j, 0) for i in range(3) for j in range(3) if (i, j) != (1, 1)],     # 48 tets, solid torus
}
TINY_CHI = {"box": 1, "block": 1, "ring": 0}


def tiny(shape: str, ns: int, seed: int, spheres=None, g: int = 18, h: float = 1.0):
    """Tiny case for the exact oracle.  ``spheres`` = (centres, radii) overrides
    the seeded random sphere set."""
    rng = np.random.default_rng(seed)
    q, tets = _cube_mesh(TINY_SHAPES[shape], h, g, rng, jitter_interior=0.15 if shape == "box" else 0.0)
    ext = q.max(axis=0) / float(1 << g)
    if spheres is None:
        c = rng.uniform(-0.1 * ext, 1.1 * ext, size=(ns, 3))
        r = rng.uniform(0.05, 0.5, size=ns) * float(ext.max())
    else:
        c, r = (np.asarray(a, dtype=np.float64) for a in spheres)
    w = _finish(f"tiny_{shape}_{ns}_{seed}", q, tets, c, r, g, 16, "fp64", expect_chi=TINY_CHI[shape])
    return w


def ring_spheres(n: int, offset=(0.013, -0.007, 0.0211), radius: float = 0.8):
    """n equal spheres around the ring's hole (at 360/n degree spacing).  The
    small offset keeps bisectors off lattice vertices."""
    th = 2 * np.pi * np.arange(n) / n + 0.05
    c = np.stack([1.5 + 1.0 * np.cos(th), 1.5 + 1.0 * np.sin(th), np.full(n, 0.5)], axis=1) + np.asarray(offset)
    return c, np.full(n, radius)


def tiny_set(count: int = 24, base_seed: int = BASE_SEED + 100):
    """Seeded tiny cases cycling through the three tiny shapes, 1-12 spheres."""
    shapes = ["box", "block", "ring"]
    out = []
    for n in range(count):
        rng = np.random.default_rng(base_seed + n)
        out.append(tiny(shapes[n % 3], int(rng.integers(1, 13)), base_seed + n))
    return out


def _thin_spheres(c, r, dmin):
    """Greedy Poisson-disk thinning in input order: keep a sphere only when
    no kept centre lies within dmin (a hash grid of cell dmin)."""
    keep, cells = [], {}
    for i, p in enumerate(c):
        key = tuple(np.floor(p / dmin).astype(np.int64))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in cells.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        if np.sum((c[j] - p) ** 2) < dmin * dmin:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            keep.append(i)
            cells.setdefault(key, []).append(i)
    keep = np.asarray(keep, dtype=np.int64)
    return c[keep], r[keep]


def batch_shapes(n: int = 32, seed: int = BASE_SEED + 5, tmin: int = 1000, tmax: int = 100_000, smin: int = 32,
                 smax: int = 4000, g: int = 19):
    """The batching workload: n seeded shapes cycling through solid tori,
    genus 0-5 slabs and ellipsoid unions, with log-uniform tet counts in
    [tmin, tmax] and sphere counts in [smin, smax] (at most one sphere per 8
    tets, for tori at most 4 per tet length along the core circle, and no two
    centres closer than 3/4 of the lattice spacing), all
    on one grid of 2^-g.  Returns a list of Workloads."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nt = float(np.exp(rng.uniform(np.log(tmin), np.log(tmax))))
        ns = int(min(np.exp(rng.uniform(np.log(smin), np.log(smax))), max(smin, nt / 8)))
        kind = i % 3
        if kind == 0:
            R, r = 1.0, rng.uniform(0.3, 0.45)
            # at least 2.5 lattice cells across the tube, or the hole is lost
            h = min((6.0 * 2 * np.pi ** 2 * R * r * r / nt) ** (1.0 / 3.0), r / 2.5)
            # core-circle spheres at most ~4 per tet length along the core,
            # so a tet meets at most a few dozen cells
            ns = min(ns, max(smin, int(4 * 2 * np.pi * R / h)))
            q, tets = lattice_mesh(torus_sdf(R, r), [-R - r - 0.05] * 2 + [-r - 0.05], [R + r + 0.05] * 2 + [r + 0.05],
                                   h, g, rng)
            c, rad = torus_core_spheres(ns, rng, R=R, rmin=0.75 * r, rmax=r)
            c, rad = _thin_spheres(c, rad, 0.75 * h)
            w = _finish(f"batch{i}_torus", q, tets, c, rad, g, 16, "fp32", expect_chi=0)
        elif kind == 1:
            m = max(2, int(round((nt / 48.0) ** (1.0 / 3.0))))
            genus = (i // 3) % 6 if m >= 8 else 0   # holes need a few cubes across
            holes = slab_holes(genus)
            q, tets = slab_mesh(BLOCK_HALF, holes, 0.2, 1.0 / m, g, rng)
            c, rad = slab_medial_spheres(ns, rng, holes, 0.2)
            c, rad = _thin_spheres(c, rad, 0.75 / m)
            w = _finish(f"batch{i}_slab{genus}", q, tets, c, rad, g, 32, "fp32", expect_chi=1 - genus)
        else:
            blob = EllipsoidBlob(int(rng.integers(6, 24)), rng)
            p = rng.uniform(blob.lo, blob.hi, size=(50000, 3))
            vol = float((blob.sdf(p) < 0).mean()) * float(np.prod(blob.hi - blob.lo))
            h = (6.0 * vol / nt) ** (1.0 / 3.0)
            q, tets = lattice_mesh(blob.sdf, blob.lo - h, blob.hi + h, h, g, rng, inside_by_vertices=True)
            c, rad = blob.medial_spheres(ns, rng)
            c, rad = _thin_spheres(c, rad, 0.75 * h)
            w = _finish(f"batch{i}_blob", q, tets, c, rad, g, 32, "fp32")
        out.append(w)
    return out


CONFIGS = {"torus_c1": torus_c1, "block_c2": block_c2, "blob_c3": blob_c3}
