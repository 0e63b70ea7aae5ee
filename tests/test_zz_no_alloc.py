"""rpd_euler_static: the no-allocation entry point gives the same chi as
rpd_build + rpd_euler, call after call.

Callers that cannot allocate device memory when they need a result (work
captured into a CUDA graph, pipelines with a fixed memory budget) use this
entry point; it takes its workspace from a fixed device array inside the
library.  Output buffers are allocated by the test beforehand, as such a
caller would do.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_18761_gb300 import build_workload, load
from paper_2403_18761_gb300.rpd import rpd_options, RPD_OK
from rpd_inputs import torus_c1

pytestmark = pytest.mark.gpu


def _static_fn():
    lib = load()
    f = lib.rpd_euler_static
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [P, I64, P, I64, P, P, I64, ctypes.POINTER(rpd_options), P, ctypes.c_int, P, P, I64,
                  ctypes.POINTER(I64)]
    f.restype = ctypes.c_int
    return lib, f


def test_static_entry_point_matches_rpd_euler_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    w = torus_c1()
    dev = torch.device("cuda")
    V = torch.as_tensor(w.verts, dtype=torch.float64, device=dev)
    T = torch.as_tensor(w.tets, dtype=torch.int32, device=dev)
    C = torch.as_tensor(w.centers, dtype=torch.float64, device=dev)
    R = torch.as_tensor(w.radii, dtype=torch.float64, device=dev)
    ctx = build_workload(w)
    want = {kind: tuple(x.cpu().numpy() for x in ctx.rpd_euler(kind)) for kind in (1, 2, 3, 4)}
    lib, f = _static_fn()
    opt = rpd_options()
    lib.rpd_default_options(ctypes.byref(opt))
    opt.precision, opt.k, opt.grid_bits = 1, w.k, w.grid_bits
    stream = torch.cuda.current_stream()
    for call in range(2):
        for kind in (1, 2, 3, 4):
            wk, wc = want[kind]
            cap = len(wc) + 8
            keys = torch.full((cap, kind), -1, dtype=torch.int32, device=dev)
            chi = torch.full((cap,), -99, dtype=torch.int32, device=dev)
            n = ctypes.c_int64(-1)
            st = f(V.data_ptr(), len(w.verts), T.data_ptr(), len(w.tets), C.data_ptr(), R.data_ptr(), len(w.radii),
                   ctypes.byref(opt), ctypes.c_void_p(stream.cuda_stream), kind, keys.data_ptr(), chi.data_ptr(), cap,
                   ctypes.byref(n))
            assert st == RPD_OK, (call, kind, st)
            assert n.value == len(wc), (call, kind, n.value, len(wc))
            m = n.value
            assert np.array_equal(keys[:m].cpu().numpy(), wk), (call, kind)
            assert np.array_equal(chi[:m].cpu().numpy(), wc), (call, kind)
    ctx.rpd_destroy()
