"""Python binding of librpd (argument marshalling only).

Every function mirrors a C entry point of ``include/rpd.h``.  PyTorch provides
device memory and the CUDA stream; all computation runs in the library's CUDA
kernels.  There is no CPU fallback: without the compiled library or a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librpd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rpd.h")

RPD_OK, RPD_E_INVALID, RPD_E_NONMANIFOLD, RPD_E_DEGENERATE = 0, 1, 2, 3
RPD_E_OOM, RPD_E_CUDA, RPD_E_OVERFLOW, RPD_E_TIMEOUT = 4, 5, 6, 7
STATUS_NAMES = {0: "RPD_OK", 1: "RPD_E_INVALID", 2: "RPD_E_NONMANIFOLD", 3: "RPD_E_DEGENERATE",
                4: "RPD_E_OOM", 5: "RPD_E_CUDA", 6: "RPD_E_OVERFLOW", 7: "RPD_E_TIMEOUT"}
RPD_CELL, RPD_FACE, RPD_EDGE, RPD_VERTEX = 1, 2, 3, 4
RPD_FP64, RPD_FP32_FILTERED = 0, 1
PRECISION = {"fp64": RPD_FP64, "fp32": RPD_FP32_FILTERED}


class RpdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rpd_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("k", ctypes.c_int32), ("grid_bits", ctypes.c_int32),
                ("debug_checks", ctypes.c_int32), ("edge_lengths", ctypes.c_int32)]


class rpd_stats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_pieces", ctypes.c_int64), ("n_records", ctypes.c_int64 * 4),
                ("n_keys", ctypes.c_int64 * 4), ("pred_fast", ctypes.c_int64), ("pred_fp64", ctypes.c_int64),
                ("pred_exact", ctypes.c_int64), ("cand_fallback", ctypes.c_int64), ("whole_tets", ctypes.c_int64),
                ("clip_vertices", ctypes.c_int64 * 3),
                ("bin_pairs", ctypes.c_int64 * 8), ("bin_cut", ctypes.c_int64 * 8), ("ms_prep", ctypes.c_float), ("ms_knn", ctypes.c_float), ("ms_cand", ctypes.c_float),
                ("ms_clip", ctypes.c_float), ("ms_finalize", ctypes.c_float * 4), ("ms_clip_kernels", ctypes.c_float),
                ("ms_clip_span", ctypes.c_float), ("update_tets", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class rpd_medial_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("vertices", "edges", "faces", "tets", "edges_thin", "faces_thin",
                                               "tets_thin", "chi", "chi_thin")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class rpd_repair_report(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("inserted", ctypes.c_int64), ("failing", ctypes.c_int64),
                ("far_samples", ctypes.c_int64), ("max_ratio", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load librpd.so (building it in-tree first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from .build import build
        build()
    lib = ctypes.CDLL(path)
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    lib.rpd_default_options.argtypes = [ctypes.POINTER(rpd_options)]
    lib.rpd_default_options.restype = None
    lib.rpd_build.argtypes = [P, I64, P, I64, P, P, I64, ctypes.POINTER(rpd_options), P, ctypes.POINTER(P)]
    lib.rpd_build.restype = ctypes.c_int
    for name in ("rpd_euler", "rpd_components", "rpd_contractible"):
        f = getattr(lib, name)
        f.argtypes = [P, ctypes.c_int, P, P, I64, ctypes.POINTER(I64)]
        f.restype = ctypes.c_int
    lib.rpd_export.argtypes = [P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_export.restype = ctypes.c_int
    lib.rpd_pieces.argtypes = [P, P, P, P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_pieces.restype = ctypes.c_int
    lib.rpd_stats_get.argtypes = [P, ctypes.POINTER(rpd_stats)]
    lib.rpd_stats_get.restype = ctypes.c_int
    lib.rpd_last_error.argtypes = [P]
    lib.rpd_last_error.restype = ctypes.c_char_p
    lib.rpd_build_error.argtypes = []
    lib.rpd_build_error.restype = ctypes.c_char_p
    lib.rpd_destroy.argtypes = [P]
    lib.rpd_destroy.restype = None
    lib.rpd_launch_count.argtypes = []
    lib.rpd_launch_count.restype = I64
    lib.rpd_peak_fma.argtypes = [ctypes.c_int32, I64, P, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.rpd_peak_fma.restype = ctypes.c_int
    lib.rpd_insert.argtypes = [P, P, P, I64]
    lib.rpd_insert.restype = ctypes.c_int
    lib.rpd_pins.argtypes = [P, ctypes.c_int, P, P, P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_pins.restype = ctypes.c_int
    lib.rpd_shrink.argtypes = [P, P, P, P, I64, P, P, P]
    lib.rpd_shrink.restype = ctypes.c_int
    lib.rpd_repair.argtypes = [P, ctypes.c_int32, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.rpd_repair.restype = ctypes.c_int
    lib.rpd_spheres.argtypes = [P, P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_spheres.restype = ctypes.c_int
    lib.rpd_edge_lengths.argtypes = [P, P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_edge_lengths.restype = ctypes.c_int
    lib.rpd_medial.argtypes = [P, ctypes.c_double, ctypes.POINTER(rpd_medial_info), P, I64, P, I64]
    lib.rpd_medial.restype = ctypes.c_int
    lib.rpd_surface_samples.argtypes = [P, P, P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_surface_samples.restype = ctypes.c_int
    lib.rpd_envelope_distance.argtypes = [P, P, I64, P, P]
    lib.rpd_envelope_distance.restype = ctypes.c_int
    lib.rpd_repair_geometry.argtypes = [P, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(rpd_repair_report)]
    lib.rpd_repair_geometry.restype = ctypes.c_int
    lib.rpd_build_batch.argtypes = [P, P, P, P, ctypes.c_int32, P, P, P, ctypes.POINTER(rpd_options), P,
                                    ctypes.POINTER(P)]
    lib.rpd_build_batch.restype = ctypes.c_int
    lib.rpd_autotune.argtypes = [P, I64, P, I64, P, P, I64, ctypes.POINTER(rpd_options), P, ctypes.c_int32,
                                 ctypes.c_int32, P, ctypes.POINTER(rpd_options), ctypes.POINTER(ctypes.c_float)]
    lib.rpd_autotune.restype = ctypes.c_int
    lib.rpd_batch_offsets.argtypes = [P, ctypes.c_int32, P]
    lib.rpd_batch_offsets.restype = ctypes.c_int
    lib.rpd_shrink_warm.argtypes = [P, P, P, P, I64, P, P, P, P, P]
    lib.rpd_shrink_warm.restype = ctypes.c_int
    lib.rpd_pin_features.argtypes = [P, P, P, P, I64, P, P]
    lib.rpd_pin_features.restype = ctypes.c_int
    lib.rpd_propose.argtypes = [P, P, P, P, I64, ctypes.c_double, P]
    lib.rpd_propose.restype = ctypes.c_int
    lib.rpd_set_proposer.argtypes = [P, P, ctypes.c_double]
    lib.rpd_set_proposer.restype = ctypes.c_int
    lib.rpd_shrink_counters.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.rpd_shrink_counters.restype = ctypes.c_int
    lib.rpd_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_uint64, P, ctypes.POINTER(P)]
    lib.rpd_mlp_create.restype = ctypes.c_int
    lib.rpd_mlp_params.argtypes = [P, P, I64, ctypes.POINTER(I64)]
    lib.rpd_mlp_params.restype = ctypes.c_int
    lib.rpd_mlp_set_params.argtypes = [P, P, I64]
    lib.rpd_mlp_set_params.restype = ctypes.c_int
    lib.rpd_mlp_forward.argtypes = [P, P, I64, P]
    lib.rpd_mlp_forward.restype = ctypes.c_int
    lib.rpd_mlp_grad.argtypes = [P, P, P, I64, P, ctypes.POINTER(ctypes.c_float)]
    lib.rpd_mlp_grad.restype = ctypes.c_int
    lib.rpd_mlp_train.argtypes = [P, P, P, I64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                  ctypes.POINTER(ctypes.c_float)]
    lib.rpd_mlp_train.restype = ctypes.c_int
    lib.rpd_mlp_destroy.argtypes = [P]
    lib.rpd_mlp_destroy.restype = None
    _lib = lib
    return lib


def rpd_launch_count():
    """Kernel launches the library has issued in this process so far."""
    return int(load().rpd_launch_count())


def rpd_peak_fma(precision, iters, stream=None):
    """Measured CUDA-core FMA peak of one precision on the current device:
    (TFLOP/s, duration of the timed launch in ms)."""
    if not torch.cuda.is_available():
        raise RuntimeError("librpd needs a CUDA device; there is no CPU fallback")
    sh, _ = _stream_handle(stream)
    tf, ms = ctypes.c_double(0), ctypes.c_double(0)
    p = PRECISION[precision] if isinstance(precision, str) else int(precision)
    st = load().rpd_peak_fma(p, int(iters), sh, ctypes.byref(tf), ctypes.byref(ms))
    if st != RPD_OK:
        raise RpdError(st, "rpd_peak_fma failed")
    return tf.value, ms.value


def header_symbols(path: str = HEADER):
    """Entry points declared in include/rpd.h."""
    with open(path) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(rpd_[a-z_]+)\s*\(", text)))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev_f64(x, dev):
    if isinstance(x, torch.Tensor) and x.dtype == torch.float64 and x.device == dev and x.is_contiguous():
        return x
    t = torch.as_tensor(x, dtype=torch.float64)
    return t.to(dev).contiguous()


def _dev_i32(x, dev):
    if isinstance(x, torch.Tensor) and x.dtype == torch.int32 and x.device == dev and x.is_contiguous():
        return x
    return torch.as_tensor(x, dtype=torch.int32).to(dev).contiguous()


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream), stream


class Ctx:
    """Owns one rpd_ctx (device workspace and results)."""

    def __init__(self, handle, stream, device, keep):
        self.handle = handle
        self.stream = stream
        self.device = device
        self._keep = keep
        self._tabs = None
        self._buf = None     # the rpd_export buffer behind the query views
        self._nkeys = None   # element counts per kind, read with the first query

    def _check(self, st):
        if st != RPD_OK:
            raise RpdError(st, load().rpd_last_error(self.handle).decode())

    def _query(self, fn, kind):
        if 1 <= kind <= 4 and self._nkeys is not None:
            return self._nkeys[kind - 1]
        n = ctypes.c_int64(0)
        self._check(fn(self.handle, kind, None, None, 0, ctypes.byref(n)))
        return n.value

    def rows_direct(self, name, kind):
        """Keys int32[n, kind] and one value per key in fresh device tensors,
        through the per-kind C entry point `name` (rpd_euler, rpd_components
        or rpd_contractible)."""
        fn = getattr(load(), name)
        n = self._query(fn, kind)
        keys = torch.empty((n, kind), dtype=torch.int32, device=self.device)
        vals = torch.empty(n, dtype=torch.uint8 if name == "rpd_contractible" else torch.int32, device=self.device)
        self._check(fn(self.handle, kind, keys.data_ptr(), vals.data_ptr(), n, None))
        return keys, vals

    def _export_all(self):
        """All element tables through one rpd_export call, as views of one
        device buffer: {kind: [keys, chi, beta0, flag]}, or the RpdError the
        per-kind entry points report for that kind."""
        lib = load()
        tabs, nk = {}, []
        for kind in (1, 2, 3, 4):
            n = ctypes.c_int64(0)
            st = lib.rpd_euler(self.handle, kind, None, None, 0, ctypes.byref(n))
            if st != RPD_OK:
                tabs[kind] = RpdError(st, lib.rpd_last_error(self.handle).decode())
            nk.append(n.value)
        self._nkeys = nk
        nb = ctypes.c_int64(0)
        self._check(lib.rpd_export(self.handle, None, 0, ctypes.byref(nb)))
        buf = torch.empty(max(nb.value, 16), dtype=torch.uint8, device=self.device)
        self._check(lib.rpd_export(self.handle, buf.data_ptr(), nb.value, None))
        self._buf = buf
        # the layout documented with rpd_export: int32 parts (each padded to
        # 16 bytes) for kinds 1..4, then the uint8 flags; split in one call
        # per region
        al = lambda x: (x + 15) & ~15
        sizes, off = [], 0
        for kind in (1, 2, 3, 4):
            m = self._nkeys[kind - 1]
            for cnt in (m * kind, m, m):
                sizes += [cnt, al(4 * cnt) // 4 - cnt]
                off += al(4 * cnt)
        foff = off
        fsizes = []
        for kind in (1, 2, 3, 4):
            m = self._nkeys[kind - 1]
            fsizes += [m, al(m) - m]
            off += al(m)
        parts = buf[:foff].view(torch.int32).split(sizes)
        flags = buf[foff:off].split(fsizes)
        for kind in (1, 2, 3, 4):
            if kind not in tabs:
                j = 6 * (kind - 1)
                tabs[kind] = [parts[j].view(-1, kind), parts[j + 2], parts[j + 4], flags[2 * (kind - 1)]]
        if off != nb.value:
            raise RuntimeError("rpd_export layout mismatch")
        return tabs

    def _table(self, kind):
        if not 1 <= kind <= 4:
            self._query(load().rpd_euler, kind)   # the C entry point reports it
        if self._tabs is None:
            self._tabs = self._export_all()
        t = self._tabs[kind]
        if isinstance(t, RpdError):
            raise t
        return t

    def tables_host(self):
        """Every element table on the host in one device-to-host copy of the
        rpd_export buffer: ({kind: (keys, chi, beta0, flag)} as numpy views of
        one pinned host buffer, bytes copied).  Kinds the build cannot report
        are left out."""
        if self._tabs is None:
            self._tabs = self._export_all()
        host = torch.empty(self._buf.numel(), dtype=torch.uint8, pin_memory=True)
        with torch.cuda.stream(self.stream):   # ordered after the export on the build's stream
            host.copy_(self._buf, non_blocking=True)
        self.stream.synchronize()
        base = self._buf.data_ptr()
        h = host.numpy()
        out = {}
        for kind, t in self._tabs.items():
            if isinstance(t, RpdError):
                continue
            views = []
            for x in t:   # the same byte ranges as the device views
                off = x.data_ptr() - base
                nbytes = x.numel() * x.element_size()
                views.append(h[off:off + nbytes].view(np.int32 if x.dtype == torch.int32 else np.uint8)
                             .reshape(tuple(x.shape)))
            out[kind] = tuple(views)
        return out, self._buf.numel()

    # The three queries return views of one buffer filled by rpd_export (the
    # keys tensor of a kind is shared by the three); rows_direct goes through
    # the per-kind entry points instead.
    def rpd_euler(self, kind):
        """(keys int32[n, kind], chi int32[n]) on the device."""
        t = self._table(kind)
        return t[0], t[1]

    def rpd_components(self, kind):
        """(keys int32[n, kind], beta0 int32[n]) on the device."""
        t = self._table(kind)
        return t[0], t[2]

    def rpd_contractible(self, kind):
        """(keys int32[n, kind], flag uint8[n]) on the device."""
        t = self._table(kind)
        return t[0], t[3]

    def rpd_pieces(self):
        """(tet int32[n], sphere int32[n], vol f64[n], moment f64[n,3]) sorted by (tet, sphere)."""
        lib = load()
        n = ctypes.c_int64(0)
        self._check(lib.rpd_pieces(self.handle, None, None, None, None, 0, ctypes.byref(n)))
        m = n.value
        t = torch.empty(m, dtype=torch.int32, device=self.device)
        s = torch.empty(m, dtype=torch.int32, device=self.device)
        v = torch.empty(m, dtype=torch.float64, device=self.device)
        mo = torch.empty((m, 3), dtype=torch.float64, device=self.device)
        self._check(lib.rpd_pieces(self.handle, _ptr(t), _ptr(s), _ptr(v), _ptr(mo), m, ctypes.byref(n)))
        return t, s, v, mo

    def rpd_insert(self, centers, radii):
        """Append spheres and update the diagram in place (partial update).
        Views handed out by earlier queries keep the old tables."""
        with torch.cuda.stream(self.stream):   # inputs staged on the context's stream
            C = _dev_f64(centers, self.device).reshape(-1, 3).contiguous()
            R = _dev_f64(radii, self.device).reshape(-1).contiguous()
            if C.shape[0] != R.shape[0]:
                raise ValueError("centers and radii differ in length")
            st = load().rpd_insert(self.handle, _ptr(C), _ptr(R), C.shape[0])
        self._check(st)
        self._keep = self._keep + (C, R)
        self._tabs = None
        self._buf = None
        self._nkeys = None

    def rpd_pins(self, kind):
        """Pins of the non-contractible elements of `kind` (1..3): (keys
        int32[n, kind], pins f64[n, 3], inward normals f64[n, 3], boundary
        faces int32[n] = 4 tet + face or -1) on the device."""
        lib = load()
        n = ctypes.c_int64(0)
        self._check(lib.rpd_pins(self.handle, kind, None, None, None, None, 0, ctypes.byref(n)))
        m = n.value
        keys = torch.empty((m, kind), dtype=torch.int32, device=self.device)
        pins = torch.empty((m, 3), dtype=torch.float64, device=self.device)
        nrm = torch.empty((m, 3), dtype=torch.float64, device=self.device)
        faces = torch.empty(m, dtype=torch.int32, device=self.device)
        if m:
            self._check(lib.rpd_pins(self.handle, kind, _ptr(keys), _ptr(pins), _ptr(nrm), _ptr(faces), m,
                                     ctypes.byref(n)))
        return keys, pins, nrm, faces

    def rpd_shrink(self, pins, normals, faces):
        """Shrunk spheres from pins: (centres f64[n, 3], radii f64[n],
        iterations int32[n]) on the device."""
        with torch.cuda.stream(self.stream):
            P = _dev_f64(pins, self.device).reshape(-1, 3).contiguous()
            N = _dev_f64(normals, self.device).reshape(-1, 3).contiguous()
            F = _dev_i32(faces, self.device).reshape(-1).contiguous()
            m = P.shape[0]
            c = torch.empty((m, 3), dtype=torch.float64, device=self.device)
            r = torch.empty(m, dtype=torch.float64, device=self.device)
            it = torch.empty(m, dtype=torch.int32, device=self.device)
            self._check(load().rpd_shrink(self.handle, _ptr(P), _ptr(N), _ptr(F), m, _ptr(c), _ptr(r), _ptr(it)))
            self.stream.synchronize()
        return c, r, it

    def shape_offsets(self, kind):
        """First row of each shape of a batch in the tables of `kind`
        (1..4; 0 for the pieces), and the total: int64[nshapes + 1]."""
        nshapes = len(self.batch["sphere_off"]) - 1 if getattr(self, "batch", None) else 1
        out = np.zeros(nshapes + 1, dtype=np.int64)
        self._check(load().rpd_batch_offsets(self.handle, int(kind), out.ctypes.data))
        return out

    def rpd_shrink_warm(self, pins, normals, faces, r_start):
        """Shrinking from proposed first radii (0 = plain start): (centres,
        radii, iterations, restarted int32[n]) on the device."""
        with torch.cuda.stream(self.stream):
            P = _dev_f64(pins, self.device).reshape(-1, 3).contiguous()
            N = _dev_f64(normals, self.device).reshape(-1, 3).contiguous()
            F = _dev_i32(faces, self.device).reshape(-1).contiguous()
            R0 = _dev_f64(r_start, self.device).reshape(-1).contiguous()
            m = P.shape[0]
            c = torch.empty((m, 3), dtype=torch.float64, device=self.device)
            r = torch.empty(m, dtype=torch.float64, device=self.device)
            it = torch.empty(m, dtype=torch.int32, device=self.device)
            rs = torch.empty(m, dtype=torch.int32, device=self.device)
            self._check(load().rpd_shrink_warm(self.handle, _ptr(P), _ptr(N), _ptr(F), m, _ptr(R0), _ptr(c), _ptr(r),
                                               _ptr(it), _ptr(rs)))
            self.stream.synchronize()
        return c, r, it, rs

    def rpd_pin_features(self, pins, normals, radii=None):
        """Proposer features f32[n, RPD_PIN_FEATURES] and, with radii, the
        targets log2(r / box diagonal) f32[n], on the device."""
        with torch.cuda.stream(self.stream):
            P = _dev_f64(pins, self.device).reshape(-1, 3).contiguous()
            N = _dev_f64(normals, self.device).reshape(-1, 3).contiguous()
            R = _dev_f64(radii, self.device).reshape(-1).contiguous() if radii is not None else None
            m = P.shape[0]
            x = torch.empty((m, RPD_PIN_FEATURES), dtype=torch.float32, device=self.device)
            t = torch.empty(m, dtype=torch.float32, device=self.device) if R is not None else None
            self._check(load().rpd_pin_features(self.handle, _ptr(P), _ptr(N), _ptr(R), m, _ptr(x), _ptr(t)))
            self.stream.synchronize()
        return (x, t) if R is not None else x

    def rpd_propose(self, mlp, pins, normals, margin=1.25):
        """First radii f64[n] proposed by the network for the pins."""
        with torch.cuda.stream(self.stream):
            P = _dev_f64(pins, self.device).reshape(-1, 3).contiguous()
            N = _dev_f64(normals, self.device).reshape(-1, 3).contiguous()
            r = torch.empty(P.shape[0], dtype=torch.float64, device=self.device)
            self._check(load().rpd_propose(self.handle, mlp.handle, _ptr(P), _ptr(N), P.shape[0], float(margin),
                                           _ptr(r)))
            self.stream.synchronize()
        return r

    def rpd_set_proposer(self, mlp, margin=1.25):
        """Use the network (None: the plain start) in the repair loops."""
        self._proposer = mlp
        self._check(load().rpd_set_proposer(self.handle, mlp.handle if mlp is not None else None, float(margin)))

    def rpd_shrink_counters(self):
        """(pins shrunk, iterations, proposals rejected) by the repair loops."""
        a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(load().rpd_shrink_counters(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def rpd_repair(self, max_rounds=64):
        """Run the topology repair loop: (rounds, spheres inserted, failing
        elements left)."""
        lib = load()
        a, b, f = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(lib.rpd_repair(self.handle, int(max_rounds), ctypes.byref(a), ctypes.byref(b), ctypes.byref(f)))
        self._tabs = None
        self._buf = None
        self._nkeys = None
        return a.value, b.value, f.value

    def rpd_spheres(self):
        """The context's spheres after grid rounding (build inputs, then
        inserted ones): (centres f64[ns, 3], radii f64[ns]) on the device."""
        lib = load()
        n = ctypes.c_int64(0)
        self._check(lib.rpd_spheres(self.handle, None, None, 0, ctypes.byref(n)))
        c = torch.empty((n.value, 3), dtype=torch.float64, device=self.device)
        r = torch.empty(n.value, dtype=torch.float64, device=self.device)
        self._check(lib.rpd_spheres(self.handle, _ptr(c), _ptr(r), n.value, ctypes.byref(n)))
        return c, r

    def rpd_edge_lengths(self):
        """(keys int32[n, 3], length f64[n]) of every restricted power edge."""
        lib = load()
        n = ctypes.c_int64(0)
        self._check(lib.rpd_edge_lengths(self.handle, None, None, 0, ctypes.byref(n)))
        k = torch.empty((n.value, 3), dtype=torch.int32, device=self.device)
        l = torch.empty(n.value, dtype=torch.float64, device=self.device)
        self._check(lib.rpd_edge_lengths(self.handle, _ptr(k), _ptr(l), n.value, ctypes.byref(n)))
        return k, l

    def rpd_medial(self, sigma):
        """Thinned dual medial mesh: (info dict, edges int32[m, 2], faces
        int32[m, 3]) on the host."""
        lib = load()
        info = rpd_medial_info()
        self._check(lib.rpd_medial(self.handle, float(sigma), ctypes.byref(info), None, 0, None, 0))
        e = np.empty((info.edges_thin, 2), dtype=np.int32)
        f = np.empty((info.faces_thin, 3), dtype=np.int32)
        self._check(lib.rpd_medial(self.handle, float(sigma), ctypes.byref(info), e.ctypes.data, len(e),
                                   f.ctypes.data, len(f)))
        return info.as_dict(), e, f

    def rpd_surface_samples(self):
        """Boundary-triangle centroids f64[n, 3], inward unit normals f64[n, 3]
        and face ids int32[n] (4 tet + face) on the device."""
        lib = load()
        n = ctypes.c_int64(0)
        self._check(lib.rpd_surface_samples(self.handle, None, None, None, 0, ctypes.byref(n)))
        p = torch.empty((n.value, 3), dtype=torch.float64, device=self.device)
        q = torch.empty((n.value, 3), dtype=torch.float64, device=self.device)
        f = torch.empty(n.value, dtype=torch.int32, device=self.device)
        self._check(lib.rpd_surface_samples(self.handle, _ptr(p), _ptr(q), _ptr(f), n.value, ctypes.byref(n)))
        return p, q, f

    def rpd_envelope_distance(self, samples):
        """Signed distance f32[n] of points to the medial mesh's envelope and
        the nearest primitive int32[n] (RPC rows, then RPF, then RPE)."""
        with torch.cuda.stream(self.stream):
            S = _dev_f64(samples, self.device).reshape(-1, 3).contiguous()
            d = torch.empty(S.shape[0], dtype=torch.float32, device=self.device)
            a = torch.empty(S.shape[0], dtype=torch.int32, device=self.device)
            self._check(load().rpd_envelope_distance(self.handle, _ptr(S), S.shape[0], _ptr(d), _ptr(a)))
            self.stream.synchronize()
        return d, a

    def rpd_repair_geometry(self, delta, max_rounds=64):
        """Repair loop with geometric preservation: the report as a dict."""
        rep = rpd_repair_report()
        self._check(load().rpd_repair_geometry(self.handle, float(delta), int(max_rounds), ctypes.byref(rep)))
        self._tabs = None
        self._buf = None
        self._nkeys = None
        return rep.as_dict()

    def rpd_stats_get(self):
        st = rpd_stats()
        self._check(load().rpd_stats_get(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def rpd_destroy(self):
        if self.handle:
            load().rpd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.rpd_destroy()
        except Exception:
            pass


def rpd_build(verts, tets, centers, radii, precision="fp32", k=16, grid_bits=20, stream=None,
              device="cuda", debug=0, edge_lengths=False) -> Ctx:
    """Build the restricted power diagram.  Inputs may be host arrays or device
    tensors; host inputs are copied to the device first."""
    if not torch.cuda.is_available():
        raise RuntimeError("librpd needs a CUDA device; there is no CPU fallback")
    lib = load()
    dev = torch.device(device)
    if dev.index is None:
        dev = torch.device(dev.type, torch.cuda.current_device())
    V = _dev_f64(verts, dev)
    T = _dev_i32(tets, dev)
    C = _dev_f64(centers, dev)
    R = _dev_f64(radii, dev)
    opt = rpd_options()
    lib.rpd_default_options(ctypes.byref(opt))
    opt.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    opt.k = int(k)
    opt.grid_bits = int(grid_bits)
    opt.debug_checks = int(debug)
    opt.edge_lengths = int(bool(edge_lengths))
    sh, stream = _stream_handle(stream)
    out = ctypes.c_void_p()
    st = lib.rpd_build(_ptr(V), V.shape[0], _ptr(T), T.shape[0], _ptr(C), _ptr(R), R.shape[0],
                       ctypes.byref(opt), sh, ctypes.byref(out))
    if st != RPD_OK:
        raise RpdError(st, lib.rpd_build_error().decode())
    return Ctx(out, stream, dev, (V, T, C, R))


def rpd_build_batch(shapes, precision="fp32", k=16, grid_bits=20, stream=None, debug=0):
    """rpd_build_batch on a list of (verts, tets, centers, radii) with
    shape-local tet indices: the arrays are concatenated and the tets
    offset (argument marshalling); returns a Ctx whose `shape_offsets(kind)`
    gives each shape's rows."""
    lib = load()
    if not torch.cuda.is_available():
        raise RuntimeError("librpd needs a CUDA device; there is no CPU fallback")
    dev = torch.device("cuda", torch.cuda.current_device())
    vs, ts, cs, rs = [], [], [], []
    voff, toff, soff = [0], [0], [0]
    for (v, t, c, r) in shapes:
        v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
        t = np.asarray(t, dtype=np.int64).reshape(-1, 4) + voff[-1]
        c = np.asarray(c, dtype=np.float64).reshape(-1, 3)
        r = np.asarray(r, dtype=np.float64).reshape(-1)
        vs.append(v), ts.append(t), cs.append(c), rs.append(r)
        voff.append(voff[-1] + len(v)), toff.append(toff[-1] + len(t)), soff.append(soff[-1] + len(r))
    V = _dev_f64(np.concatenate(vs), dev)
    T = _dev_i32(np.concatenate(ts).astype(np.int32), dev)
    C = _dev_f64(np.concatenate(cs), dev)
    R = _dev_f64(np.concatenate(rs), dev)
    hv, ht, hs = (np.asarray(o, dtype=np.int64) for o in (voff, toff, soff))
    opt = rpd_options()
    lib.rpd_default_options(ctypes.byref(opt))
    opt.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    opt.k = int(k)
    opt.grid_bits = int(grid_bits)
    opt.debug_checks = int(debug)
    sh, stream = _stream_handle(stream)
    out = ctypes.c_void_p()
    st = lib.rpd_build_batch(_ptr(V), _ptr(T), _ptr(C), _ptr(R), len(shapes), hv.ctypes.data, ht.ctypes.data,
                             hs.ctypes.data, ctypes.byref(opt), sh, ctypes.byref(out))
    if st != RPD_OK:
        raise RpdError(st, lib.rpd_build_error().decode())
    ctx = Ctx(out, stream, dev, (V, T, C, R))
    ctx.batch = dict(vert_off=hv, tet_off=ht, sphere_off=hs)
    return ctx


def rpd_autotune(verts, tets, centers, radii, ks=(8, 16, 24, 32), reps=3, precision="fp32", grid_bits=20,
                 stream=None):
    """The library's autotuner: (fastest k, its median build time in ms)."""
    lib = load()
    if not torch.cuda.is_available():
        raise RuntimeError("librpd needs a CUDA device; there is no CPU fallback")
    dev = torch.device("cuda", torch.cuda.current_device())
    V, T, C, R = _dev_f64(verts, dev), _dev_i32(tets, dev), _dev_f64(centers, dev), _dev_f64(radii, dev)
    base = rpd_options()
    lib.rpd_default_options(ctypes.byref(base))
    base.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    base.grid_bits = int(grid_bits)
    kk = np.asarray(ks, dtype=np.int32)
    best = rpd_options()
    ms = ctypes.c_float(0)
    sh, _ = _stream_handle(stream)
    st = lib.rpd_autotune(_ptr(V), V.shape[0], _ptr(T), T.shape[0], _ptr(C), _ptr(R), R.shape[0], ctypes.byref(base),
                          kk.ctypes.data, len(kk), int(reps), sh, ctypes.byref(best), ctypes.byref(ms))
    if st != RPD_OK:
        raise RpdError(st, lib.rpd_build_error().decode())
    return int(best.k), float(ms.value)


def build_workload(w, precision=None, k=None, stream=None, debug=0, edge_lengths=False):
    """rpd_build on a seeded workload (see rpd_inputs)."""
    return rpd_build(w.verts, w.tets, w.centers, w.radii, precision=precision or w.precision,
                     k=k or w.k, grid_bits=w.grid_bits, stream=stream, debug=debug, edge_lengths=edge_lengths)


def collect(ctx):
    """All outputs of a context as host numpy arrays (for tests and checks)."""
    out = {"kinds": {}}
    for kind in (RPD_CELL, RPD_FACE, RPD_EDGE, RPD_VERTEX):
        keys, chi = ctx.rpd_euler(kind)
        _, beta = ctx.rpd_components(kind)
        _, flag = ctx.rpd_contractible(kind)
        out["kinds"][kind] = dict(keys=keys.cpu().numpy(), chi=chi.cpu().numpy(), beta0=beta.cpu().numpy(),
                                  flag=flag.cpu().numpy())
    t, s, v, m = ctx.rpd_pieces()
    out.update(tet=t.cpu().numpy(), sphere=s.cpu().numpy(), vol=v.cpu().numpy(), moment=m.cpu().numpy())
    out["stats"] = ctx.rpd_stats_get()
    return out


RPD_PIN_FEATURES = 30
MLP_NPARAM = 37377


class Mlp:
    """Owns one rpd_mlp: the learned radius proposer (3 x 128 ReLU layers on
    the tensor cores, BF16 operands, FP32 master weights, Adam)."""

    def __init__(self, n_in=RPD_PIN_FEATURES, seed=0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("librpd needs a CUDA device; there is no CPU fallback")
        sh, self.stream = _stream_handle(stream)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.n_in = int(n_in)
        h = ctypes.c_void_p()
        st = load().rpd_mlp_create(self.n_in, int(seed), sh, ctypes.byref(h))
        if st != RPD_OK:
            raise RpdError(st, "rpd_mlp_create failed")
        self.handle = h

    def _check(self, st, what):
        if st != RPD_OK:
            raise RpdError(st, what + " failed")

    def _x(self, x):
        x = torch.as_tensor(x, dtype=torch.float32).to(self.device).reshape(-1, self.n_in).contiguous()
        return x

    def params(self):
        p = torch.empty(MLP_NPARAM, dtype=torch.float32, device=self.device)
        self._check(load().rpd_mlp_params(self.handle, _ptr(p), MLP_NPARAM, None), "rpd_mlp_params")
        return p

    def set_params(self, p):
        p = torch.as_tensor(p, dtype=torch.float32).to(self.device).reshape(-1).contiguous()
        self._check(load().rpd_mlp_set_params(self.handle, _ptr(p), p.numel()), "rpd_mlp_set_params")

    def forward(self, x):
        x = self._x(x)
        y = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        self._check(load().rpd_mlp_forward(self.handle, _ptr(x), x.shape[0], _ptr(y)), "rpd_mlp_forward")
        return y

    def grad(self, x, t):
        """(gradient f32[37377] of mean((y - t)^2), loss)."""
        x = self._x(x)
        t = torch.as_tensor(t, dtype=torch.float32).to(self.device).reshape(-1).contiguous()
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=self.device)
        loss = ctypes.c_float(0)
        self._check(load().rpd_mlp_grad(self.handle, _ptr(x), _ptr(t), x.shape[0], _ptr(g), ctypes.byref(loss)),
                    "rpd_mlp_grad")
        return g, loss.value

    def train(self, x, t, steps, batch=1024, lr=1e-3):
        """Adam steps on consecutive batches of the rows; the last loss."""
        x = self._x(x)
        t = torch.as_tensor(t, dtype=torch.float32).to(self.device).reshape(-1).contiguous()
        loss = ctypes.c_float(0)
        self._check(load().rpd_mlp_train(self.handle, _ptr(x), _ptr(t), x.shape[0], int(steps), int(batch),
                                         float(lr), ctypes.byref(loss)), "rpd_mlp_train")
        return loss.value

    def destroy(self):
        if self.handle:
            load().rpd_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
