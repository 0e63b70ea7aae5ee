"""Seeded synthetic inputs: tetrahedral meshes and medial-sphere sets.

Shared by the tests, the oracle checks and the benchmark.  Holds none of the
restricted-power-diagram arithmetic.
"""
from .configs import (Workload, torus_c1, block_c2, blob_c3, genus_slab, batch_shapes, tiny, tiny_set,
                      ring_spheres, CONFIGS, BASE_SEED)
from .mesh import validate, face_adjacency, snap

__all__ = ["Workload", "torus_c1", "block_c2", "blob_c3", "genus_slab", "batch_shapes", "tiny", "tiny_set", "ring_spheres",
           "CONFIGS", "BASE_SEED", "validate", "face_adjacency", "snap"]
