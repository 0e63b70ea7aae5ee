"""Analytic shapes and seeded medial-sphere samplers (input generator only).

Each shape has a signed distance function ``sdf(x)`` (negative inside) used to
carve the lattice mesh, and a sampler that places spheres near the shape's
medial axis with radius equal to the distance to the boundary, in the spirit of
the paper's medial spheres (Sec. 3.1).  Nothing here computes any part of the
restricted power diagram.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------- solid torus
def torus_sdf(R: float, r: float):
    def f(x):
        x = np.asarray(x, dtype=np.float64)
        q = np.hypot(x[..., 0], x[..., 1]) - R
        return np.hypot(q, x[..., 2]) - r
    return f


def torus_core_spheres(n: int, rng: np.random.Generator, R: float = 1.0,
                       sigma: float = 0.02, rmin: float = 0.3, rmax: float = 0.4,
                       phase: float = 0.1234):
    """Centres on the core circle plus N(0, sigma^2) jitter, radii U(rmin, rmax)."""
    th = 2.0 * np.pi * np.arange(n) / n + phase
    c = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(n)], axis=1)
    c = c + rng.normal(0.0, sigma, size=c.shape)
    rad = rng.uniform(rmin, rmax, size=n)
    return c, rad


# ------------------------------------------------- genus-3 block (CAD-like)
BLOCK_HALF = np.array([2.0, 1.0, 0.5])
HOLES_X = (-1.2, 0.0, 1.2)
HOLE_R = 0.3


def _block_prims(x):
    """Distances from interior points to each primitive surface: 6 box planes
    and 3 z-through cylinders.  Shape (..., 9)."""
    x = np.asarray(x, dtype=np.float64)
    d = [BLOCK_HALF[a] - x[..., a] for a in range(3)] + [BLOCK_HALF[a] + x[..., a] for a in range(3)]
    for cx in HOLES_X:
        d.append(np.hypot(x[..., 0] - cx, x[..., 1]) - HOLE_R)
    return np.stack(d, axis=-1)


def block_sdf(x):
    return -_block_prims(x).min(axis=-1)


def block_medial_spheres(n: int, rng: np.random.Generator, tol: float = 0.02):
    """Rejection-sample interior points whose two nearest primitives are within
    ``tol`` of each other (near-medial); radius = distance to the boundary."""
    out = []
    total = 0
    while total < n:
        p = rng.uniform(-BLOCK_HALF, BLOCK_HALF, size=(65536, 3))
        d = _block_prims(p)
        ok = d.min(axis=-1) > 0
        ds = np.sort(d, axis=-1)
        ok &= (ds[:, 1] - ds[:, 0]) < tol
        p = p[ok]
        out.append(np.concatenate([p, ds[ok][:, :1]], axis=1))
        total += len(p)
    s = np.concatenate(out, axis=0)[:n]
    return s[:, :3].copy(), s[:, 3].copy()


# ------------------------------------------- slabs of genus g (repair loop)
def slab_holes(genus: int):
    """x positions of `genus` z-through holes of radius HOLE_R spread along
    the 4x2x1 slab (genus 0: no hole)."""
    if genus <= 0:
        return ()
    return tuple(float(v) for v in np.linspace(-1.3, 1.3, genus)) if genus > 1 else (0.0,)


def _slab_prims(x, holes, hole_r):
    x = np.asarray(x, dtype=np.float64)
    d = [BLOCK_HALF[a] - x[..., a] for a in range(3)] + [BLOCK_HALF[a] + x[..., a] for a in range(3)]
    for cx in holes:
        d.append(np.hypot(x[..., 0] - cx, x[..., 1]) - hole_r)
    return np.stack(d, axis=-1)


def slab_sdf(holes, hole_r):
    return lambda x: -_slab_prims(x, holes, hole_r).min(axis=-1)


def slab_medial_spheres(n: int, rng: np.random.Generator, holes, hole_r, tol: float = 0.02):
    """Near-medial interior samples of the slab with holes (two nearest
    primitives within `tol`); radius = distance to the boundary."""
    out = []
    total = 0
    while total < n:
        p = rng.uniform(-BLOCK_HALF, BLOCK_HALF, size=(65536, 3))
        d = _slab_prims(p, holes, hole_r)
        ok = d.min(axis=-1) > 0
        ds = np.sort(d, axis=-1)
        ok &= (ds[:, 1] - ds[:, 0]) < tol
        p = p[ok]
        out.append(np.concatenate([p, ds[ok][:, :1]], axis=1))
        total += len(p)
    s = np.concatenate(out, axis=0)[:n]
    return s[:, :3].copy(), s[:, 3].copy()


# ------------------------------------------------------ organic ellipsoid blob
def random_rotations(n: int, rng: np.random.Generator):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], axis=1)


class EllipsoidBlob:
    """Union of ellipsoids with axes U(amin, amax), random rotations and centres
    from a seeded random walk (consecutive centres overlap, so the union is
    connected).  The signed distance is approximated per ellipsoid by the scaled
    radial distance (|D^-1 R^T (x-m)| - 1) * min(axes)."""

    def __init__(self, n: int, rng: np.random.Generator, amin: float = 0.1, amax: float = 0.5,
                 step: float = 0.25):
        self.axes = rng.uniform(amin, amax, size=(n, 3))
        self.rot = random_rotations(n, rng)
        c = np.zeros((n, 3))
        for k in range(1, n):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            c[k] = c[rng.integers(0, k)] + step * d
        self.centers = c - c.mean(axis=0)
        rad = self.axes.max(axis=1)
        self.lo = (self.centers - rad[:, None]).min(axis=0)
        self.hi = (self.centers + rad[:, None]).max(axis=0)

    def sdf(self, x, chunk: int = 4096):
        """Approximate signed distance; batched over all ellipsoids with torch
        (CPU, every host core) in float64."""
        import torch
        x = np.asarray(x, dtype=np.float64)
        shp = x.shape[:-1]
        xt = torch.from_numpy(np.ascontiguousarray(x.reshape(-1, 3)))
        c = torch.from_numpy(self.centers)                    # (E, 3)
        r = torch.from_numpy(np.ascontiguousarray(self.rot))  # (E, 3, 3)
        inv_a = torch.from_numpy(1.0 / self.axes)              # (E, 3)
        amin = torch.from_numpy(self.axes.min(axis=1))         # (E,)
        out = torch.empty(xt.shape[0], dtype=torch.float64)
        for s in range(0, xt.shape[0], chunk):
            d = xt[s:s + chunk][None, :, :] - c[:, None, :]      # (E, n, 3)
            y = torch.bmm(d, r) * inv_a[:, None, :]
            g = (torch.linalg.vector_norm(y, dim=2) - 1.0) * amin[:, None]
            out[s:s + chunk] = g.min(dim=0).values
        return out.numpy().reshape(shp)

    def medial_spheres(self, n: int, rng: np.random.Generator, eps: float = 0.01, gmax: float = 0.6):
        """Interior points where the finite-difference gradient of the depth is
        small (ridge of the distance field); radius = depth."""
        out = []
        total = 0
        while total < n:
            p = rng.uniform(self.lo, self.hi, size=(16384, 3))
            dep = -self.sdf(p)
            p, dep = p[dep > 0.02], dep[dep > 0.02]
            if len(p) == 0:
                continue
            g2 = np.zeros(len(p))
            for a in range(3):
                e = np.zeros(3)
                e[a] = eps
                g2 += ((self.sdf(p + e) - self.sdf(p - e)) / (2 * eps)) ** 2
            ok = np.sqrt(g2) < gmax
            out.append(np.concatenate([p[ok], dep[ok][:, None]], axis=1))
            total += int(ok.sum())
        s = np.concatenate(out, axis=0)[:n]
        return s[:, :3].copy(), s[:, 3].copy()
