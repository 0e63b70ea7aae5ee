"""Recovery paths of rpd_build on the GPU: a rebuild after the element-record
buffers overflow, and a clean failure when a device allocation fails.

Both are driven from the host through the library's test hooks
(RPD_RECORD_CAP: capacity of the first record buffers; RPD_PAIR_CAP: room of
the binning done before the pair count is known; RPD_FAIL_ALLOC_AFTER: the
allocation that fails); none touches the device in an unsafe way.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2403_18761_gb300 import build_workload
from paper_2403_18761_gb300.rpd import collect
from rpd_inputs import torus_c1

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _same(a, b):
    for kind in (1, 2, 3, 4):
        for f in ("keys", "chi", "beta0", "flag"):
            assert np.array_equal(a["kinds"][kind][f], b["kinds"][kind][f]), (kind, f)
    for f in ("tet", "sphere", "vol", "moment"):
        assert np.array_equal(a[f], b[f]), f


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_record_overflow_rebuilds_identically(precision):
    w = torus_c1()
    ctx = build_workload(w, precision=precision)
    want = collect(ctx)
    ctx.rpd_destroy()
    os.environ["RPD_RECORD_CAP"] = "64"   # far below the element records of this mesh
    try:
        ctx = build_workload(w, precision=precision)
        got = collect(ctx)
        ctx.rpd_destroy()
    finally:
        del os.environ["RPD_RECORD_CAP"]
    assert all(got["stats"]["n_records"][k] > 64 for k in (1, 2)), got["stats"]["n_records"]
    _same(got, want)


def test_pair_binning_overflow_bins_again():
    """With room for far fewer pairs than there are, the binning done before
    the pair count is read drops its excess writes and is redone with room for
    all pairs; results are identical."""
    w = torus_c1()
    ctx = build_workload(w, precision="fp32")
    want = collect(ctx)
    ctx.rpd_destroy()
    os.environ["RPD_PAIR_CAP"] = "100"
    try:
        ctx = build_workload(w, precision="fp32")
        got = collect(ctx)
        ctx.rpd_destroy()
    finally:
        del os.environ["RPD_PAIR_CAP"]
    assert got["stats"]["n_pairs"] > 100
    _same(got, want)


_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
from paper_2403_18761_gb300 import build_workload, RpdError
from paper_2403_18761_gb300.rpd import RPD_E_OOM
from rpd_inputs import torus_c1
w = torus_c1()
fails = 0
try:
    build_workload(w)
except RpdError as e:
    fails = 1
    assert e.status == RPD_E_OOM, e.status
print("FAILED_CLEANLY" if fails else "NO_FAILURE")
"""


@pytest.mark.parametrize("after", [3, 25, 60])
def test_allocation_failure_is_reported(after):
    env = dict(os.environ, RPD_FAIL_ALLOC_AFTER=str(after))
    out = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "FAILED_CLEANLY" in out.stdout, out.stdout


# ------------------------------------------------- bounded waits run out
# Each case runs in a child process: the hook makes one bounded device loop
# give up (a wait on a row that no tile publishes; a union-find bound of 0),
# the build must return RPD_E_TIMEOUT with the context still usable, and the
# next build, with the hook removed, must match the oracle.
_TIMEOUT_CHILD = r"""
import os, sys
sys.path.insert(0, {root!r})
import numpy as np
import oracle
from paper_2403_18761_gb300 import build_workload, RpdError
from paper_2403_18761_gb300.rpd import RPD_E_TIMEOUT, collect
from rpd_inputs import block_c2
w = block_c2(h=0.12, ns=300)   # 5.8k mesh vertices: two tiles in the vertex sort
os.environ[{var!r}] = {val!r}
try:
    build_workload(w, precision="fp32", debug={debug})
    print("NO_TIMEOUT")
    sys.exit(0)
except RpdError as e:
    assert e.status == RPD_E_TIMEOUT, e
    print("TIMEOUT:", e)
del os.environ[{var!r}]
g = collect(build_workload(w, precision="fp32", debug={debug}))
o = oracle.run(w)
assert np.array_equal(g["tet"], o["tet"]) and np.array_equal(g["sphere"], o["sphere"])
for kind in (1, 2, 3, 4):
    for f in ("keys", "chi", "beta0"):
        assert np.array_equal(g["kinds"][kind][f], o["kinds"][kind][f].astype(np.int32)), (kind, f)
print("RECOVERED")
"""


@pytest.mark.parametrize("var,val,debug", [("RPD_TEST_LOOKBACK_STALL", "4096", 4), ("RPD_TEST_UF_LIMIT", "0", 0)])
def test_bounded_wait_runs_out_and_next_build_is_correct(var, val, debug):
    code = _TIMEOUT_CHILD.format(root=ROOT, var=var, val=val, debug=debug)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    assert "TIMEOUT:" in out.stdout and "RECOVERED" in out.stdout, out.stdout
