"""rpd_euler_static: the no-allocation entry point gives the same chi as
rpd_build + rpd_euler, call after call.

Callers that cannot allocate device memory when they need a result
(pipelines with a fixed device-memory budget, services that must not
allocate while they run) use this entry point; it takes its workspace from a
fixed device array inside the library.  Output buffers are allocated by the
test beforehand, as such a caller would do.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_18761_gb300 import build_workload, load
from paper_2403_18761_gb300.rpd import rpd_options, RPD_OK, RPD_E_OVERFLOW, RPD_E_INVALID
from rpd_inputs import torus_c1, block_c2

pytestmark = pytest.mark.gpu


def _static_fn():
    lib = load()
    f = lib.rpd_euler_static
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [P, I64, P, I64, P, P, I64, ctypes.POINTER(rpd_options), P, ctypes.c_int, P, P, I64,
                  ctypes.POINTER(I64)]
    f.restype = ctypes.c_int
    return lib, f


def _device_inputs(w, dev):
    return (torch.as_tensor(w.verts, dtype=torch.float64, device=dev),
            torch.as_tensor(w.tets, dtype=torch.int32, device=dev),
            torch.as_tensor(w.centers, dtype=torch.float64, device=dev),
            torch.as_tensor(w.radii, dtype=torch.float64, device=dev))


def _call(f, w, ins, opt, kind, keys=None, chi=None, cap=0):
    V, T, C, R = ins
    n = ctypes.c_int64(-1)
    st = f(V.data_ptr(), len(w.verts), T.data_ptr(), len(w.tets), C.data_ptr(), R.data_ptr(), len(w.radii),
           ctypes.byref(opt), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), kind,
           keys.data_ptr() if keys is not None else None, chi.data_ptr() if chi is not None else None, cap,
           ctypes.byref(n))
    return st, n.value


def _options(lib, w, precision):
    opt = rpd_options()
    lib.rpd_default_options(ctypes.byref(opt))
    opt.precision, opt.k, opt.grid_bits = precision, w.k, w.grid_bits
    return opt


def _check_matches(f, w, ins, opt, want, dev, tag):
    for kind in (1, 2, 3, 4):
        wk, wc = want[kind]
        st, n = _call(f, w, ins, opt, kind)   # count only: NULL outputs
        assert st == RPD_OK and n == len(wc), (tag, kind, st, n)
        cap = len(wc) + 8
        keys = torch.full((cap, kind), -1, dtype=torch.int32, device=dev)
        chi = torch.full((cap,), -99, dtype=torch.int32, device=dev)
        st, n = _call(f, w, ins, opt, kind, keys, chi, cap)
        assert st == RPD_OK, (tag, kind, st)
        assert n == len(wc), (tag, kind, n, len(wc))
        assert np.array_equal(keys[:n].cpu().numpy(), wk), (tag, kind)
        assert np.array_equal(chi[:n].cpu().numpy(), wc), (tag, kind)
        assert bool((chi[n:] == -99).all()), (tag, kind)   # nothing written past n


@pytest.mark.parametrize("precision", [1, 0])
def test_static_entry_point_matches_rpd_euler_twice(precision):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    w = torus_c1()
    dev = torch.device("cuda")
    ins = _device_inputs(w, dev)
    ctx = build_workload(w, precision="fp32" if precision == 1 else "fp64")
    want = {kind: tuple(x.cpu().numpy() for x in ctx.rpd_euler(kind)) for kind in (1, 2, 3, 4)}
    ctx.rpd_destroy()
    lib, f = _static_fn()
    opt = _options(lib, w, precision)
    for call in range(2):
        _check_matches(f, w, ins, opt, want, dev, (precision, call))


def test_static_entry_point_rejects_what_does_not_fit_and_recovers():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda")
    lib, f = _static_fn()
    small = torus_c1()
    ins = _device_inputs(small, dev)
    ctx = build_workload(small, precision="fp32")
    want = {kind: tuple(x.cpu().numpy() for x in ctx.rpd_euler(kind)) for kind in (1, 2, 3, 4)}
    ctx.rpd_destroy()
    opt = _options(lib, small, 1)
    # a 200k-tet problem needs far more than the fixed array holds
    big = block_c2()
    big_ins = _device_inputs(big, dev)
    st, _ = _call(f, big, big_ins, _options(lib, big, 1), 1)
    assert st == RPD_E_OVERFLOW, st
    # cap smaller than the element count, and an unknown precision
    keys = torch.empty((4, 2), dtype=torch.int32, device=dev)
    chi = torch.empty(4, dtype=torch.int32, device=dev)
    st, n = _call(f, small, ins, opt, 2, keys, chi, 4)
    assert st == RPD_E_INVALID and n == len(want[2][1]), (st, n)
    bad = _options(lib, small, 7)
    assert _call(f, small, ins, bad, 1)[0] == RPD_E_INVALID
    # the shared array serves the next call correctly
    _check_matches(f, small, ins, opt, want, dev, "after rejections")
