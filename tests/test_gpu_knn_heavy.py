"""The neighbour search's heavy-sphere list (debug bit 8: the largest weights
kept out of the grid and scanned first by every vertex) must not change
anything: the tables and pieces with it equal those without it, on an
organic blob with a heavy-tailed radius distribution and on the block."""
import numpy as np
import pytest
import torch

from paper_2403_18761_gb300 import build_workload
from paper_2403_18761_gb300.rpd import collect
from rpd_inputs import blob_c3, block_c2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


@pytest.mark.parametrize("make", [lambda: blob_c3(target_tets=60_000, ns=3000, n_ellipsoids=40),
                                  lambda: block_c2(h=0.1, ns=1500)])
def test_heavy_list_changes_nothing(make):
    w = make()
    a = collect(build_workload(w))
    b = collect(build_workload(w, debug=8))
    for kind in (1, 2, 3, 4):
        for f in ("keys", "chi", "beta0", "flag"):
            assert np.array_equal(a["kinds"][kind][f], b["kinds"][kind][f]), (kind, f)
    for f in ("tet", "sphere", "vol", "moment"):
        assert np.array_equal(a[f], b[f]), f
    # a tighter completeness bound can only spare fallback searches
    assert b["stats"]["cand_fallback"] <= a["stats"]["cand_fallback"]
