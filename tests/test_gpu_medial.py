"""Dual medial mesh and thinning (Sec. 3.2, Sec. 5.3) through the C-ABI.

* RPE lengths (computed in the volume pass, summed per key in fixed point)
  against the oracle's segment lengths.
* The library's thinning against the CPU restatement (oracle/thin.py) fed
  with the same tables and importances.
* The nerve theorem (Thm. 1): once every element is contractible the medial
  mesh has the shape's Euler characteristic, and thinning keeps it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.thin import thin
from paper_2403_18761_gb300 import build_workload
from paper_2403_18761_gb300.rpd import collect
from rpd_inputs import torus_c1, block_c2, tiny, ring_spheres
from rpd_inputs.configs import Workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    oracle.build()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", ["torus", "block"])
def test_edge_lengths_match_oracle(case, precision):
    w = torus_c1() if case == "torus" else block_c2(h=0.15, ns=300)
    ctx = build_workload(w, precision=precision, edge_lengths=True)
    keys, length = (x.cpu().numpy() for x in ctx.rpd_edge_lengths())
    o = oracle.run(w)["kinds"][3]
    assert np.array_equal(keys, o["keys"].astype(np.int32))
    want = o["length"] / float(1 << w.grid_bits)
    diam = float(np.linalg.norm(w.verts.max(axis=0) - w.verts.min(axis=0)))
    assert np.all(np.abs(length - want) <= 1e-9 * want + 1e-12 * diam), np.max(np.abs(length - want))


def _tables(ctx, w):
    g = collect(ctx)
    k3, l3 = (x.cpu().numpy() for x in ctx.rpd_edge_lengths())
    c, r = (x.cpu().numpy() for x in ctx.rpd_spheres())
    alpha = {tuple(int(v) for v in k): float(l) / (2.0 * r[k].sum() / 3.0) for k, l in zip(k3, l3)}
    edges = [tuple(int(v) for v in k) for k in g["kinds"][2]["keys"]]
    faces = [tuple(int(v) for v in k) for k in g["kinds"][3]["keys"]]
    tets = [tuple(int(v) for v in k) for k in g["kinds"][4]["keys"]]
    return g, edges, faces, tets, alpha


@pytest.mark.parametrize("sigma", [0.1, 0.3, 10.0])
def test_thinning_matches_cpu_restatement(sigma):
    w = block_c2(h=0.15, ns=300)
    ctx = build_workload(w, edge_lengths=True)
    g, edges, faces, tets, alpha = _tables(ctx, w)
    info, e, f = ctx.rpd_medial(sigma)
    assert info["vertices"] == len(g["kinds"][1]["keys"]) and info["tets"] == len(tets)
    we, wf, wt = thin(edges, faces, alpha, tets, sigma)
    assert [tuple(x) for x in e.tolist()] == we
    assert [tuple(x) for x in f.tolist()] == wf
    assert info["tets_thin"] == len(wt)
    assert info["chi_thin"] == info["chi"]


def test_nerve_theorem_after_repair():
    """Thm. 1: all RPC/RPF/RPE contractible -> the medial mesh (the nerve) is
    homotopy equivalent to the shape: chi(medial) = chi(torus) = 0, and
    thinning removes every tetrahedron without changing it."""
    w = torus_c1()
    sub = Workload(w.name, w.verts, w.tets, w.centers[::16], w.radii[::16], w.grid_bits, w.k, w.precision, w.info)
    ctx = build_workload(sub, edge_lengths=True)
    _, _, failing = ctx.rpd_repair(64)
    assert failing == 0
    info, e, f = ctx.rpd_medial(0.3)
    assert info["chi"] == w.info["chi"] == 0
    assert info["chi_thin"] == 0 and info["tets_thin"] == 0


def test_edge_lengths_need_the_build_option():
    from paper_2403_18761_gb300 import RpdError
    from paper_2403_18761_gb300.rpd import RPD_E_INVALID
    ctx = build_workload(torus_c1())
    with pytest.raises(RpdError) as e:
        ctx.rpd_edge_lengths()
    assert e.value.status == RPD_E_INVALID
    with pytest.raises(RpdError):
        ctx.rpd_medial(0.3)
