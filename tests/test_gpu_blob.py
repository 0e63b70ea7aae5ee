"""The organic-blob workload at full size (union of 200 seeded ellipsoids,
~2.0 M tets, 20,000 near-medial spheres, k = 32): parity with the C oracle on
a seeded 1% tet sample (the oracle's pieces stored by
tests/golden/make_golden.py), invariants that hold at any size, and the
FP32-filtered and FP64 predicate modes agreeing."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_18761_gb300 import build_workload
from paper_2403_18761_gb300.rpd import collect
from rpd_inputs import blob_c3

from test_gpu_parity import _check_pieces, _tet_geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def blob():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    oracle.build()
    w = blob_c3()
    return w, collect(build_workload(w, precision="fp32"))


def test_blob_sampled_tets_match_oracle(blob):
    import hashlib
    import os
    w, g = blob
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "blob_c3_sample.npz"))
    h = hashlib.sha256()
    for a in (w.verts, w.tets, w.centers, w.radii):
        h.update(np.ascontiguousarray(a).tobytes())
    assert h.hexdigest() == str(ref["input_digest"]), "the blob generator changed: rerun make_golden.py"
    sub = ref["sample"]
    assert len(sub) >= 0.01 * w.nt - 1
    _check_pieces(w, g, ref["tet"], ref["sphere"], ref["vol"], ref["moment"], sel=sub)


def test_blob_invariants(blob):
    w, g = blob
    vol, _, _ = _tet_geometry(w)
    per = np.bincount(g["tet"], weights=g["vol"], minlength=w.nt)
    assert np.all(np.abs(per - vol) <= 1e-12 * vol)
    tot = sum((-1) ** (k - 1) * int(d["chi"].sum()) for k, d in g["kinds"].items())
    assert tot == w.info["chi"]
    for d in g["kinds"].values():
        k = d["keys"]
        if k.shape[1] > 1:
            assert np.all(np.diff(k, axis=1) > 0)
        assert np.all(np.diff(k[:, 0]) >= 0)
        assert np.all(d["beta0"] >= 1)
        assert np.array_equal(d["flag"].astype(bool), (d["beta0"] == 1) & (d["chi"] == 1))


def test_blob_precisions_agree(blob):
    w, g = blob
    h = collect(build_workload(w, precision="fp64"))
    assert np.array_equal(h["tet"], g["tet"]) and np.array_equal(h["sphere"], g["sphere"])
    for kind in (1, 2, 3, 4):
        for f in ("keys", "chi", "beta0", "flag"):
            assert np.array_equal(h["kinds"][kind][f], g["kinds"][kind][f]), (kind, f)
    assert np.max(np.abs(h["vol"] - g["vol"])) <= 1e-12 * np.max(g["vol"])
