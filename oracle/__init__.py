"""CPU oracle for the restricted power diagram (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import, call or link anything under ``oracle/``.  The library under
``paper_2403_18761_gb300/`` never does and has no CPU fallback.

Two tiers, sharing no code with the CUDA library:

* ``oracle.tiny``      exact rationals (Python ``fractions``), any dimension,
                       for inputs of a few dozen simplices; pins the rules.
* ``oracle.run``       plain C brute force (``rpd_oracle.c``): FP64
                       construction, exact 256-bit predicates, every tet
                       clipped against every other sphere; aggregated here with
                       numpy and scipy.

``run(w, k=K)`` runs the same C clipping on per-tet candidate sets found by
the library's neighbour + candidate algorithm (restated in C in the same file,
no code shared with the library).  It is the benchmark's same-algorithm CPU
baseline, not a parity reference; a CPU test checks it against the brute force.

Per-key aggregation (this file):
  chi(key)   = sum of the per-piece fractional contributions (Sec. 4.1.2);
  length     = summed segment lengths of an edge element (grid units), the
               RPE length in the thinning's importance (Sec. 5.3);
  beta0(key) = connected components of the key's pieces linked across shared
               tet faces (Sec. 4.1.1);
  flag(key)  = beta0 == 1 and chi == 1 (Sec. 3.3, Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librpd_oracle.so")
_lib = None

STATUS = {0: "OK", 1: "INVALID", 2: "NONMANIFOLD", 3: "DEGENERATE", 4: "OOM", 6: "OVERFLOW"}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no GPU needed)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_run.restype = P
        lib.orc_run.argtypes = [I64, P, I64, P, I64, P, P, P, I64, ctypes.c_int]
        lib.orc_run_knn.restype = P
        lib.orc_run_knn.argtypes = [I64, P, I64, P, I64, P, P, P, I64, ctypes.c_int, ctypes.c_int]
        lib.orc_status.restype = ctypes.c_int
        lib.orc_status.argtypes = [P]
        lib.orc_npieces.restype = I64
        lib.orc_npieces.argtypes = [P]
        lib.orc_nnodes.restype = I64
        lib.orc_nnodes.argtypes = [P]
        lib.orc_copy.restype = None
        lib.orc_copy.argtypes = [P] * 12 + [I64, P]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [P]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {STATUS.get(status, status)}")
        self.status = status


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def clip_all(verts_i, tets, centers_i, radii_i, subset=None, nthreads=None, k=0):
    """Run the C brute force (k = 0) or the same-algorithm baseline with k
    power neighbours per vertex.  Integer grid inputs.  Returns raw pieces and
    element nodes (unsorted) and the face adjacency."""
    lib = _load()
    X = np.ascontiguousarray(verts_i, dtype=np.int64)
    T = np.ascontiguousarray(tets, dtype=np.int32)
    C = np.ascontiguousarray(centers_i, dtype=np.int64)
    R = np.ascontiguousarray(radii_i, dtype=np.int64)
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
    nth = nthreads or os.cpu_count() or 1
    args = (len(X), _ptr(X), len(T), _ptr(T), len(R), _ptr(C), _ptr(R), _ptr(sub), 0 if sub is None else len(sub), nth)
    h = lib.orc_run_knn(*args, int(k)) if k else lib.orc_run(*args)
    try:
        st = lib.orc_status(h)
        if st != 0:
            raise OracleError(st)
        np_, nn = lib.orc_npieces(h), lib.orc_nnodes(h)
        out = dict(p_t=np.empty(np_, np.int32), p_i=np.empty(np_, np.int32), p_vol=np.empty(np_),
                   p_mom=np.empty((np_, 3)), n_kind=np.empty(nn, np.int32), n_key=np.empty((nn, 4), np.int32),
                   n_t=np.empty(nn, np.int32), n_own=np.empty(nn, np.int32), n_link=np.empty(nn, np.int32),
                   n_frac=np.empty(nn), adj=np.empty((len(T), 4), np.int32), n_len=np.empty(nn))
        lib.orc_copy(h, *[_ptr(out[k]) for k in ("p_t", "p_i", "p_vol", "p_mom", "n_kind", "n_key", "n_t",
                                                 "n_own", "n_link", "n_frac", "adj")], len(T), _ptr(out["n_len"]))
    finally:
        lib.orc_free(h)
    out["nthreads"] = nth
    return out


def aggregate(raw, nt):
    """Per-kind sorted keys with chi (owner rule), chi (1/n rule) and beta0."""
    res = {}
    kinds = raw["n_kind"]
    for kind in (1, 2, 3, 4):
        sel = np.nonzero(kinds == kind)[0]
        keys = raw["n_key"][sel, :kind].astype(np.int64)
        tt = raw["n_t"][sel].astype(np.int64)
        if len(sel) == 0:
            res[kind] = dict(keys=np.zeros((0, kind), np.int64), chi=np.zeros(0, np.int64),
                             chi_frac=np.zeros(0), beta0=np.zeros(0, np.int64), length=np.zeros(0))
            continue
        ukeys, kid = np.unique(keys, axis=0, return_inverse=True)
        kid = kid.ravel()
        chi = np.bincount(kid, weights=raw["n_own"][sel], minlength=len(ukeys)).round().astype(np.int64)
        chi_frac = np.bincount(kid, weights=raw["n_frac"][sel], minlength=len(ukeys))
        length = np.bincount(kid, weights=raw["n_len"][sel], minlength=len(ukeys))   # edges: segment lengths
        # components: node (kid, t) linked to (kid, adj[t][f]) for each link bit f
        comp = kid * nt + tt
        order = np.argsort(comp, kind="stable")
        scomp = comp[order]
        rows, cols = [], []
        for f in range(4):
            has = (raw["n_link"][sel] >> f) & 1
            src = np.nonzero(has)[0]
            t2 = raw["adj"][tt[src], f].astype(np.int64)
            q = kid[src] * nt + t2
            pos = np.searchsorted(scomp, q)
            ok = (pos < len(scomp)) & (scomp[np.minimum(pos, len(scomp) - 1)] == q)
            if not ok.all():
                raise AssertionError("component link target missing")
            rows.append(src)
            cols.append(order[pos])
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        g = coo_matrix((np.ones(len(rows), np.int8), (rows, cols)), shape=(len(sel), len(sel)))
        _, lab = connected_components(g, directed=False)
        pairs = np.unique(np.stack([kid, lab], axis=1), axis=0)
        beta0 = np.bincount(pairs[:, 0], minlength=len(ukeys)).astype(np.int64)
        res[kind] = dict(keys=ukeys, chi=chi, chi_frac=chi_frac, beta0=beta0, length=length)
    return res


def run(w, subset=None, nthreads=None, k=0):
    """Oracle RPD of a seeded workload: pieces (sorted by (tet, sphere)) in
    world units and, unless ``subset`` is given, per-key chi / beta0 / flags.
    k > 0 selects the same-algorithm CPU baseline (k power neighbours)."""
    q, c, r = w.ints()
    t0 = time.perf_counter()
    raw = clip_all(q, w.tets, c, r, subset=subset, nthreads=nthreads, k=k)
    elapsed = time.perf_counter() - t0
    s = 1.0 / float(1 << w.grid_bits)
    order = np.lexsort((raw["p_i"], raw["p_t"]))
    out = dict(tet=raw["p_t"][order], sphere=raw["p_i"][order], vol=raw["p_vol"][order] * s ** 3,
               moment=raw["p_mom"][order] * s ** 4, seconds=elapsed, nthreads=raw["nthreads"], raw=raw)
    if subset is None:
        agg = aggregate(raw, len(w.tets))
        for kind, d in agg.items():
            d["flag"] = (d["beta0"] == 1) & (d["chi"] == 1)
        out["kinds"] = agg
    return out
