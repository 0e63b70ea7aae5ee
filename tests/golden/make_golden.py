"""Writes the stored expected values of the full-size parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``rpd_inputs/``); nothing here touches the CUDA library.

* ``block_c2_full.npz``: the genus-3 block workload (204,782 tets, 2,000
  spheres) run through the brute-force oracle in full: every element table
  (keys, chi, beta0 per kind), the nonempty piece list (tet, sphere) as a
  SHA-256 digest plus its length, and the volume and first moment of every
  restricted power cell (sums over its pieces).
* ``blob_c3_sample.npz``: the organic-blob workload (union of 200 ellipsoids,
  ~2.0M tets, 20,000 spheres) on a seeded 1% tet sample: the sample, and the
  sample's pieces (tet, sphere, volume, first moment).

Each file also stores a digest of the workload's inputs, so that a test can
tell a changed generator from a wrong result.

    python tests/golden/make_golden.py [block_c2] [blob_c3]
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from rpd_inputs import block_c2, blob_c3  # noqa: E402

BLOB_SAMPLE_SEED = 20240320
BLOB_SAMPLE_FRACTION = 0.01


def input_digest(w):
    h = hashlib.sha256()
    for a in (w.verts, w.tets, w.centers, w.radii):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def piece_digest(tet, sphere):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(tet, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(sphere, dtype=np.int32).tobytes())
    return h.hexdigest()


def blob_sample(nt):
    rng = np.random.default_rng(BLOB_SAMPLE_SEED)
    n = int(round(BLOB_SAMPLE_FRACTION * nt))
    return np.sort(rng.choice(nt, size=n, replace=False)).astype(np.int32)


def make_block():
    w = block_c2()
    t0 = time.time()
    o = oracle.run(w)
    out = dict(input_digest=np.array(input_digest(w)), pieces_digest=np.array(piece_digest(o["tet"], o["sphere"])),
               n_pieces=np.array(len(o["tet"])))
    ns = w.ns
    out["cell_vol"] = np.bincount(o["sphere"], weights=o["vol"], minlength=ns)
    for a in range(3):
        out[f"cell_mom{a}"] = np.bincount(o["sphere"], weights=o["moment"][:, a], minlength=ns)
    for kind in (1, 2, 3, 4):
        d = o["kinds"][kind]
        out[f"keys{kind}"] = d["keys"].astype(np.int32)
        out[f"chi{kind}"] = d["chi"].astype(np.int32)
        out[f"beta{kind}"] = d["beta0"].astype(np.int32)
    np.savez_compressed(os.path.join(HERE, "block_c2_full.npz"), **out)
    print(f"block_c2: {len(o['tet'])} pieces in {time.time() - t0:.1f} s", flush=True)


def make_blob():
    w = blob_c3()
    sub = blob_sample(w.nt)
    t0 = time.time()
    o = oracle.run(w, subset=sub)
    np.savez_compressed(os.path.join(HERE, "blob_c3_sample.npz"), input_digest=np.array(input_digest(w)),
                        sample=sub, tet=o["tet"], sphere=o["sphere"], vol=o["vol"], moment=o["moment"])
    print(f"blob_c3: {len(sub)} tets, {len(o['tet'])} pieces in {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["block_c2", "blob_c3"]
    oracle.build()
    if "block_c2" in which:
        make_block()
    if "blob_c3" in which:
        make_blob()
