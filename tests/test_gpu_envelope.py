"""Geometric preservation (Sec. 4.3) through the C-ABI: the distance of surface
samples to the medial mesh's enveloping volume against the CPU restatement
(oracle/envelope.py) on the oracle's own element tables, and the repair loop
with the geometric threshold.

FP32 arithmetic in the kernel (the distance only decides a threshold): the
bar is |d_gpu - d_cpu| <= 2e-5 x the bounding-box diagonal.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.envelope import envelope_distance
from paper_2403_18761_gb300 import build_workload
from rpd_inputs import torus_c1, block_c2, genus_slab
from rpd_inputs.configs import Workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    oracle.build()


def _cpu_distance(w, S):
    o = oracle.run(w)["kinds"]
    q, c, r = w.ints()
    sc = 1.0 / float(1 << w.grid_bits)
    C = c.astype(np.float64) * sc
    R = r.astype(np.float64) * sc
    e = [tuple(k) for k in o[2]["keys"].tolist()]
    f = [tuple(k) for k in o[3]["keys"].tolist()]
    return envelope_distance(S, C, R, e, f, vertices=o[1]["keys"][:, 0])


@pytest.mark.parametrize("case", ["torus", "block"])
def test_envelope_distance_matches_cpu(case):
    w = torus_c1() if case == "torus" else block_c2(h=0.15, ns=300)
    ctx = build_workload(w)
    P, N, F = (x.cpu().numpy() for x in ctx.rpd_surface_samples())
    rng = np.random.default_rng(2)
    lo, hi = w.verts.min(axis=0), w.verts.max(axis=0)
    S = np.concatenate([P[rng.choice(len(P), 160, replace=False)], rng.uniform(lo, hi, (80, 3))])
    d, a = (x.cpu().numpy() for x in ctx.rpd_envelope_distance(S))
    want = _cpu_distance(w, S)
    diag = float(np.linalg.norm(hi - lo))
    assert np.all(a >= 0)
    assert np.max(np.abs(d - want)) <= 2e-5 * diag, np.max(np.abs(d - want))


def test_geometric_repair_bounds_the_distance():
    """A genus-1 slab from 16 near-medial spheres: topology repaired, then
    every surface sample within delta x diagonal of the envelope (checked
    again on the CPU for a sample of them)."""
    w = genus_slab(1, h=0.15, ns=16)
    ctx = build_workload(w)
    delta = 0.02
    rep = ctx.rpd_repair_geometry(delta, 64)
    assert rep["failing"] == 0 and rep["far_samples"] == 0, rep
    assert rep["max_ratio"] <= delta
    P, _, _ = (x.cpu().numpy() for x in ctx.rpd_surface_samples())
    diag = float(np.linalg.norm(P.max(axis=0) - P.min(axis=0)))
    c, r = (x.cpu().numpy() for x in ctx.rpd_spheres())
    fin = Workload(w.name, w.verts, w.tets, c, r, w.grid_bits, w.k, w.precision, w.info)
    rng = np.random.default_rng(5)
    S = P[rng.choice(len(P), 120, replace=False)]
    assert np.max(_cpu_distance(fin, S)) <= delta * diag + 2e-5 * diag
