"""Benchmark: restricted (tet, sphere) pieces per second, including the
fractional Euler characteristic, connected components and contractibility of
every RPC/RPF/RPE/RPV, on one GB300.

One step = rpd_build + rpd_euler/rpd_components/rpd_contractible for every
element kind (all of the hot path) on the organic-blob workload (union of 200
seeded ellipsoids, ~2.0M tets, 20k near-medial spheres, k = 32), FP32-filtered
clipping with FP64/exact fallback, compared on the same step with the plain
FP64 form and with the volumes of the CPU oracle on a tet sample.  Inputs are
seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config blob_c3|block_c2|torus_c1] [--precision fp32|fp64]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "restricted (tet,sphere) pieces/sec incl. Euler+components; FP32-filtered vs FP64"
UNIT = "pieces/s"
WORKLOADS = {
    "block_c2": "genus-3 block 4x2x1 with 3 through-holes, ~200k tets, 2000 near-medial spheres, k=32",
    "torus_c1": "solid torus R=1 r=0.4, ~5k tets, 64 core-circle spheres, k=16",
    "blob_c3": "union of 200 ellipsoids, ~2M tets, 20000 near-medial spheres, k=32",
}


# Algorithmic FP32 work per nonempty piece of the clip stage, as planned for
# Tet-Cell clipping (Sec. 5.2) with k power neighbours: per clip V_cur x (7 flop
# for the sign test + 7 for its bound) plus ~60 per constructed vertex, about
# 2.5 kFLOP at k = 16 and 4.5 kFLOP at k = 32.  This is the roofline's
# `achieved` numerator (flop per piece x pieces of the step).
PLANNED_FLOP_PER_PIECE = {16: 2500.0, 32: 4500.0}
# The work the kernels execute is far smaller, because each piece is clipped
# only by its tet's few candidate spheres and the error bound is stored with
# the vertex: one filtered sign test F.C is 3 FMA + 1 MUL = 7 flop; a vertex
# constructed on a new plane takes the cofactors of its m radical-plane rows
# (m = 1: a selection, 0 flop; m = 2: three 2x2 minors, 9 flop; m = 3: four
# 3x3 cofactors, 56 flop) plus its orientation test and stored bound (17).
FLOP_SIGN_TEST = 7
FLOP_NEW_VERTEX = (17, 26, 73)   # by m = 1, 2, 3
# DRAM bytes (read + write) per step of the clip kernels (k_clip over all bins
# + k_whole), from one ncu capture of the current kernels per workload and
# precision; a workload missing here reports traffic null.
CLIP_TRAFFIC_BYTES = {("blob_c3", "fp32"): 894.12e6}
# CPU legs per workload, sized for 10-30 s each on the 16 host cores: tets of
# the brute-force oracle sample, of its 1-thread sample, fraction of tets for
# the same-algorithm baseline, tets per step of the reference arm.
CPU_SAMPLES = {
    "blob_c3": dict(oracle=500, oracle_1t=24, fair=0.25, ref=200),
    "block_c2": dict(oracle=10000, oracle_1t=600, fair=1.0, ref=2000),
    "torus_c1": dict(oracle=5051, oracle_1t=2000, fair=1.0, ref=5051),
}


def job_throughput(local_ms, local_units, world, device="cpu"):
    """Whole-job throughput of N replicas: the timed region is the slowest
    rank's (max over ranks of its summed step times) and every rank processed
    local_units (weak scaling: the same workload per rank).  Returns
    (max time in ms, units per second over all ranks)."""
    import torch
    import torch.distributed as dist
    total_ms = float(local_ms)
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    return total_ms, local_units * world / (total_ms / 1e3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def fma_peaks(target_ms=300.0, repeats=3):
    """FP32 and FP64 CUDA-core peaks from the library's FMA-chain
    microbenchmark (rpd_peak_fma): a short probe sizes each run to about
    target_ms; the best of `repeats` runs is kept."""
    from paper_2403_18761_gb300 import rpd_peak_fma
    out = {}
    for prec in ("fp32", "fp64"):
        probe_iters = 1 << 12
        _, ms = rpd_peak_fma(prec, probe_iters)
        iters = max(probe_iters, int(probe_iters * target_ms / max(ms, 1e-3)))
        best, best_ms = 0.0, 0.0
        for _ in range(repeats):
            tf, ms = rpd_peak_fma(prec, iters)
            if tf > best:
                best, best_ms = tf, ms
        out[prec] = {"tflops": best, "ms": best_ms, "iters": iters}
    return out


def counted_flop(s):
    """FP32 (or FP64) flop the clip kernels execute for one step's counters."""
    tests = s["pred_fast"] + s["pred_fp64"] + s["pred_exact"]
    nv = s["clip_vertices"]
    return FLOP_SIGN_TEST * max(tests - sum(nv), 0) + sum(f * n for f, n in zip(FLOP_NEW_VERTEX, nv))


def clip_roofline(stage, k, workload, precision, peaks, hbm_gbs, stage64=None):
    """Roofline of the clip kernels (the dominant kernel family): CUDA-core
    ALU bound.  `achieved` = planned flop per piece x pieces / the clip-kernel
    span timed by the library's CUDA events on the launching streams; the
    FP32, FP64 and HBM fractions use the measured peaks."""
    kk = min(PLANNED_FLOP_PER_PIECE, key=lambda q: abs(q - k))
    pieces = float(np.mean([s["n_pieces"] for s in stage]))
    ms = float(np.mean([s["ms_clip_kernels"] for s in stage]))
    flop_planned = PLANNED_FLOP_PER_PIECE[kk] * pieces
    flop_exec = float(np.mean([counted_flop(s) for s in stage]))
    p32, p64 = peaks["fp32"]["tflops"], peaks["fp64"]["tflops"]
    peak = p32 if precision == "fp32" else p64
    achieved = flop_planned / (ms * 1e-3) / 1e12
    traffic = CLIP_TRAFFIC_BYTES.get((workload, precision))
    fr = {"fp32" if precision == "fp32" else "fp64": achieved / peak,
          (precision + "_executed"): flop_exec / (ms * 1e-3) / 1e12 / peak}
    if traffic is not None and hbm_gbs:
        fr["hbm"] = traffic / (ms * 1e-3) / 1e9 / hbm_gbs
    out = {"kernel": "k_clip over all candidate-count bins + k_whole (side by side on the bin streams; "
                     "timed to the end of the record kernels that follow them there)",
           "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": traffic, "flop_per_launch": flop_planned, "flop_per_piece": PLANNED_FLOP_PER_PIECE[kk],
           "flop_executed_per_launch": flop_exec, "achieved_executed": flop_exec / (ms * 1e-3) / 1e12,
           "ms_per_launch": ms,
           "peak_source": f"measured: rpd_peak_fma {precision} FMA chains (of measured)",
           "fractions": fr}
    if stage64:
        ms64 = float(np.mean([s["ms_clip_kernels"] for s in stage64]))
        f64 = PLANNED_FLOP_PER_PIECE[kk] * float(np.mean([s["n_pieces"] for s in stage64]))
        fr["fp64_mode_fp64"] = f64 / (ms64 * 1e-3) / 1e12 / p64
        fr["fp64_mode_fp64_executed"] = float(np.mean([counted_flop(s) for s in stage64])) / (ms64 * 1e-3) / 1e12 / p64
    # the resource closest to its peak, judged on executed work: the planned
    # count assumes every candidate clips every piece and overstates the
    # FP64 mode, where the filter's early exits do not apply
    named = {k: v for k, v in fr.items() if k in (precision + "_executed", "hbm", "fp64_mode_fp64_executed")}
    out["binding"] = max(named, key=named.get)
    return out


def make_workload(name):
    import rpd_inputs
    return rpd_inputs.CONFIGS[name]()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _sample(nt, n, seed):
    rng = np.random.default_rng(seed)
    n = max(1, min(int(n), nt))
    return np.sort(rng.choice(nt, size=n, replace=False)).astype(np.int32)


def cpu_baselines(w, config, seed=20240318):
    """The CPU legs, each on a seeded tet sample of the workload (sizes in
    CPU_SAMPLES): the brute-force oracle as it stands on all host cores and on
    one thread, and the same-algorithm baseline (the library's neighbour +
    candidate algorithm restated in C in the oracle's file, FP64 + exact
    predicates) on all host cores.  Returns (cpu_baseline, extra legs,
    (sample, oracle result)) where the oracle result serves the volume error."""
    import oracle
    oracle.build()
    cfg = CPU_SAMPLES.get(config, CPU_SAMPLES["block_c2"])
    sub = _sample(w.nt, cfg["oracle"], seed)
    t0 = time.perf_counter()
    o = oracle.run(w, subset=sub)
    dt = time.perf_counter() - t0
    base = dict(value=len(o["tet"]) / dt, unit=UNIT, cores=o["nthreads"], kind="oracle",
                sample=f"{len(sub)} of {w.nt} tets (seed {seed}), all {w.ns} spheres, brute-force C oracle; "
                       f"{len(o['tet'])} pieces in {dt:.2f} s")
    legs = {}
    sub1 = _sample(w.nt, cfg["oracle_1t"], seed + 1)
    t0 = time.perf_counter()
    o1 = oracle.run(w, subset=sub1, nthreads=1)
    dt = time.perf_counter() - t0
    legs["oracle_1thread"] = dict(value=len(o1["tet"]) / dt, unit=UNIT, cores=1, kind="oracle",
                                  sample=f"{len(sub1)} tets (seed {seed + 1}); {len(o1['tet'])} pieces in {dt:.2f} s")
    frac = cfg["fair"]
    subf = None if frac >= 1.0 else _sample(w.nt, frac * w.nt, seed + 2)
    t0 = time.perf_counter()
    of = oracle.run(w, subset=subf, k=w.k)
    dt = time.perf_counter() - t0
    legs["same_algorithm"] = dict(value=len(of["tet"]) / dt, unit=UNIT, cores=of["nthreads"],
                                  kind="same kNN + candidate algorithm, C, FP64 + exact predicates",
                                  sample=(f"all {w.nt} tets" if subf is None else f"{len(subf)} of {w.nt} tets "
                                          f"({100 * frac:.0f}%, seed {seed + 2})") +
                                  f", k = {w.k}; {len(of['tet'])} pieces in {dt:.2f} s (pieces and elements "
                                  "equal the brute force's, checked by the CPU tests)")
    return base, legs, (sub, o)


def volume_error(w, pieces, sub, o):
    """Volume and first-moment error of the GPU pieces of the sampled tets
    against the oracle, relative to the tet's volume (moments: volume x
    diameter, about the tet centroid)."""
    gt, gs, gv, gm = pieces
    keep = np.isin(gt, sub)
    gt, gs, gv, gm = gt[keep], gs[keep], gv[keep], gm[keep]
    if not (np.array_equal(gt, o["tet"]) and np.array_equal(gs, o["sphere"])):
        return {"pieces_match": False}
    q, _, _ = w.ints()
    sc = 1.0 / float(1 << w.grid_bits)
    P = q[w.tets[gt].astype(np.int64)].astype(np.float64) * sc
    a, b, c = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]
    vt = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    cen = P.mean(axis=1)
    diam = np.max(np.linalg.norm(P[:, :, None, :] - P[:, None, :, :], axis=-1), axis=(1, 2))
    ev = np.abs(gv - o["vol"]) / vt
    em = np.linalg.norm((gm - gv[:, None] * cen) - (o["moment"] - o["vol"][:, None] * cen), axis=1) / (vt * diam)
    return {"pieces_match": True, "pieces": int(len(gv)), "volume_max": float(ev.max(initial=0)),
            "volume_median": float(np.median(ev)) if len(ev) else 0.0, "moment_max": float(em.max(initial=0)),
            "relative_to": "tet volume (moment: tet volume x diameter)"}


def batch_leg(nshapes, steps, warmup, stream, flush, dev, seed=20240323):
    """Batching (many shapes of uneven size): the same seeded shapes built
    one rpd_build per shape in a loop, and as one rpd_build_batch, each step
    with the 12 table queries per build; the batch's k chosen by the
    library's autotuner first.  Device time by CUDA events on the stream."""
    import torch
    from paper_2403_18761_gb300 import rpd_build
    from paper_2403_18761_gb300.rpd import load, rpd_options, PRECISION, _ptr
    import ctypes
    import rpd_inputs
    ws = rpd_inputs.batch_shapes(nshapes, seed=seed)
    g = ws[0].grid_bits
    dshapes = [tuple(torch.as_tensor(a, dtype=dt, device=dev) for a, dt in
                     zip((w.verts, w.tets, w.centers, w.radii), (torch.float64, torch.int32, torch.float64,
                                                                 torch.float64))) for w in ws]

    def queries(ctx):
        for kind in (1, 2, 3, 4):
            ctx.rpd_euler(kind), ctx.rpd_components(kind), ctx.rpd_contractible(kind)

    def timed(fn):
        out = []
        with torch.cuda.stream(stream):
            for it in range(warmup + steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pieces = fn()
                e1.record(stream)
                e1.synchronize()
                if it >= warmup:
                    out.append(e0.elapsed_time(e1))
        return float(np.mean(out)), pieces

    # the autotuner on the batch (k only: the clip tiles follow the candidate counts)
    lib = load()
    hv = np.cumsum([0] + [len(w.verts) for w in ws]).astype(np.int64)
    ht = np.cumsum([0] + [len(w.tets) for w in ws]).astype(np.int64)
    hs = np.cumsum([0] + [len(w.radii) for w in ws]).astype(np.int64)
    V = torch.as_tensor(np.concatenate([w.verts for w in ws]), dtype=torch.float64, device=dev)
    T = torch.as_tensor(np.concatenate([w.tets + o for w, o in zip(ws, hv[:-1])]), dtype=torch.int32, device=dev)
    C = torch.as_tensor(np.concatenate([w.centers for w in ws]), dtype=torch.float64, device=dev)
    R = torch.as_tensor(np.concatenate([w.radii for w in ws]), dtype=torch.float64, device=dev)
    base = rpd_options()
    lib.rpd_default_options(ctypes.byref(base))
    base.precision, base.grid_bits = PRECISION["fp32"], g
    ks = np.asarray([8, 16, 24, 32], dtype=np.int32)
    best, tms = rpd_options(), ctypes.c_float(0)
    st = lib.rpd_autotune_batch(_ptr(V), _ptr(T), _ptr(C), _ptr(R), len(ws), hv.ctypes.data, ht.ctypes.data,
                                hs.ctypes.data, ctypes.byref(base), ks.ctypes.data, len(ks), 2,
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(best), ctypes.byref(tms))
    if st != 0:
        return {"shapes": len(ws), "error": f"rpd_autotune_batch returned {st}: "
                                            f"{lib.rpd_build_error().decode()}"}
    k = int(best.k)

    def loop():
        n = 0
        for (v, t, c, r) in dshapes:
            ctx = rpd_build(v, t, c, r, precision="fp32", k=k, grid_bits=g, stream=stream)
            queries(ctx)
            n += ctx.rpd_stats_get()["n_pieces"]
            ctx.rpd_destroy()
        return n

    def batched():
        from paper_2403_18761_gb300.rpd import Ctx
        out = ctypes.c_void_p()
        opt = rpd_options()
        lib.rpd_default_options(ctypes.byref(opt))
        opt.precision, opt.grid_bits, opt.k = PRECISION["fp32"], g, k
        s = lib.rpd_build_batch(_ptr(V), _ptr(T), _ptr(C), _ptr(R), len(ws), hv.ctypes.data, ht.ctypes.data,
                                hs.ctypes.data, ctypes.byref(opt), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(out))
        if s != 0:
            raise RuntimeError(f"rpd_build_batch failed ({s})")
        ctx = Ctx(out, stream, dev, (V, T, C, R))
        queries(ctx)
        n = ctx.rpd_stats_get()["n_pieces"]
        ctx.rpd_destroy()
        return n

    ms_loop, p_loop = timed(loop)
    ms_batch, p_batch = timed(batched)
    return {"shapes": len(ws), "tets": int(ht[-1]), "spheres": int(hs[-1]),
            "workload": f"{len(ws)} seeded tori / genus 0-5 slabs / ellipsoid unions, log-uniform 1k-100k tets, "
                        f"32-4k spheres (at most one per 8 tets)",
            "k_autotuned": k, "autotune_ms_best": float(tms.value), "pieces_per_step": int(p_batch),
            "pieces_equal": bool(p_loop == p_batch),
            "per_shape_loop": {"ms_per_step": ms_loop, "value": p_loop / (ms_loop * 1e-3), "unit": UNIT},
            "batched": {"ms_per_step": ms_batch, "value": p_batch / (ms_batch * 1e-3), "unit": UNIT},
            "batched_over_loop": ms_loop / ms_batch}


TRAIN_STEPS, TRAIN_BATCH = 1000, 8192   # the proposer's training in the repair leg


def repair_leg(nshapes, stream, dev, seed=20240330):
    """The topology-repair workload: seeded genus 0-5 slabs (~125k tets, 256
    near-medial starting spheres) repaired by rpd_repair, plain and with the
    learned radius proposer (trained first by the library's own kernels on
    the (pin features -> shrunk radius) pairs of ten other slabs); wall time
    per shape on the host clock (the loop synchronises every round)."""
    import torch
    from paper_2403_18761_gb300 import build_workload, Mlp
    import rpd_inputs
    train = [rpd_inputs.genus_slab(g, seed=seed + 1 + s, h=0.075, ns=64) for g in (0, 1, 2, 4, 5) for s in (0, 1)]
    xs, ts = [], []
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for w in train:
            ctx = build_workload(w, stream=stream)
            P, N, F = ctx.rpd_surface_samples()
            _, r, _ = ctx.rpd_shrink(P, N, F)
            x, t = ctx.rpd_pin_features(P, N, r)
            keep = torch.isfinite(t)
            xs.append(x[keep])
            ts.append(t[keep])
            ctx.rpd_destroy()
        x, t = torch.cat(xs), torch.cat(ts)
        perm = torch.randperm(x.shape[0], generator=torch.Generator().manual_seed(0)).to(dev)
        x, t = x[perm].contiguous(), t[perm].contiguous()
        net = Mlp(seed=7, stream=stream)
        _, l0 = net.grad(x, t)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.train(x, t, steps=TRAIN_STEPS, batch=TRAIN_BATCH, lr=1e-3)
        e1.record(stream)
        e1.synchronize()
        _, l1 = net.grad(x, t)
    train_ms = e0.elapsed_time(e1)
    # tensor-core work of training: per row, the three hidden layers'
    # forward GEMMs (32x128, 128x128, 128x128), their weight gradients (the
    # same flops) and the input gradients of layers 2 and 1
    gemm_flop = TRAIN_STEPS * TRAIN_BATCH * 2.0 * (2 * (32 * 128 + 2 * 128 * 128) + 2 * 128 * 128)
    bf16_peak = measured_peaks().get("bf16_tflops")
    mlp_tf = gemm_flop / (train_ms * 1e-3) / 1e12
    shapes = []
    for g in range(nshapes):
        w = rpd_inputs.genus_slab(g % 6, seed=seed + 100 + g, h=0.075, ns=256)
        row = {"genus": g % 6, "tets": int(w.nt)}
        for mode in ("plain", "learned"):
            with torch.cuda.stream(stream):
                ctx = build_workload(w, stream=stream)
                if mode == "learned":
                    ctx.rpd_set_proposer(net, 1.25)
                torch.cuda.synchronize()
                a = time.perf_counter()
                rounds, inserted, failing = ctx.rpd_repair(96)
                b = time.perf_counter()
                pins, iters, rej = ctx.rpd_shrink_counters()
                ctx.rpd_destroy()
            row[mode] = {"ms": (b - a) * 1e3, "rounds": rounds, "inserted": inserted, "failing": failing,
                         "shrink_pins": pins, "shrink_iters": iters, "rejected": rej}
        shapes.append(row)
    summary = repair_summary(shapes)
    return {"workload": f"{nshapes} genus 0-5 slabs 4x2x1 (~125k tets each), 256 near-medial starting spheres",
            "training": {"pairs": int(x.shape[0]), "steps": TRAIN_STEPS, "batch": TRAIN_BATCH, "loss_before": l0,
                         "loss_after": l1, "train_ms": train_ms,
                         "roofline": {"bound": "tensor", "achieved": mlp_tf, "unit": "TFLOP/s",
                                      "peak": bf16_peak, "frac": (mlp_tf / bf16_peak) if bf16_peak else None,
                                      "flop": gemm_flop,
                                      "note": "tcgen05 BF16 GEMMs of 128-row tiles (one CTA each), 15 kernels "
                                              "per step replayed from a CUDA graph; latency-bound at this batch"},
                         "setup_s": time.perf_counter() - t0},
            **summary}


def repair_summary(shapes):
    """Per-shape repair rows ({"genus", "tets", "plain": {...}, "learned":
    {...}}) summed: over the shapes both arms brought to all-contractible,
    over all, and per genus; the shapes left with failing elements listed."""
    modes = ("plain", "learned")
    keys = ("ms", "rounds", "inserted", "failing", "shrink_pins", "shrink_iters", "rejected")

    def total(rows):
        return {m: {k: sum(r[m][k] for r in rows) for k in keys} for m in modes}

    done = [r for r in shapes if r["plain"]["failing"] == 0 and r["learned"]["failing"] == 0]
    stalled = [dict(r, index=i) for i, r in enumerate(shapes)
               if r["plain"]["failing"] or r["learned"]["failing"]]
    by_genus = {}
    for g in sorted({r["genus"] for r in shapes}):
        rows = [r for r in shapes if r["genus"] == g]
        by_genus[str(g)] = dict(total(rows), shapes=len(rows),
                                repaired=sum(1 for r in rows if r["plain"]["failing"] == 0),
                                needed_repair=sum(1 for r in rows if r["plain"]["rounds"] > 0))
    return {"shapes": len(shapes), "repaired": len(done), "by_genus": by_genus,
            "total_repaired": total(done), "total": total(shapes), "stalled": stalled,
            "same_result": all(r["plain"]["inserted"] == r["learned"]["inserted"] and
                               r["plain"]["failing"] == r["learned"]["failing"] for r in shapes)}


def medial_envelope_leg(w, precision, kk, stream, dev, steps=3):
    """The dual medial mesh and its thinning (Sec. 3.2, 5.3) and the
    geometric check (Sec. 4.3) on the headline workload: a build that also
    measures the RPE lengths, rpd_medial (sigma 0.1, organic shapes), and the
    envelope distance of every boundary-triangle centroid to the spheres,
    cones and slabs.  Device times by CUDA events on the stream; the thinning
    is a host process (its wall time)."""
    import torch
    from paper_2403_18761_gb300 import rpd_build
    V = torch.as_tensor(w.verts, dtype=torch.float64, device=dev)
    T = torch.as_tensor(w.tets, dtype=torch.int32, device=dev)
    C = torch.as_tensor(w.centers, dtype=torch.float64, device=dev)
    R = torch.as_tensor(w.radii, dtype=torch.float64, device=dev)
    out = {}
    with torch.cuda.stream(stream):
        ms_len, ms_env, s_thin = [], [], []
        for it in range(steps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx = rpd_build(V, T, C, R, precision=precision, k=kk, grid_bits=w.grid_bits, stream=stream,
                            edge_lengths=True)
            e1.record(stream)
            e1.synchronize()
            a = time.perf_counter()
            info, _, _ = ctx.rpd_medial(0.1)
            b = time.perf_counter()
            P, N, F = ctx.rpd_surface_samples()
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            d, prim = ctx.rpd_envelope_distance(P)
            f1.record(stream)
            f1.synchronize()
            if it > 0:
                ms_len.append(e0.elapsed_time(e1))
                ms_env.append(f0.elapsed_time(f1))
                s_thin.append(b - a)
            nsamp = int(P.shape[0])
            diag = float(torch.linalg.norm(P.max(dim=0).values - P.min(dim=0).values))
            dd = d.double() / diag
            ctx.rpd_destroy()
    nprim = info["vertices"] + info["edges"] + info["faces"]
    out["medial"] = {"build_with_edge_lengths_ms": float(np.mean(ms_len)), "thinning_s": float(np.mean(s_thin)),
                     "sigma": 0.1, "info": info}
    out["envelope"] = {"samples": nsamp, "primitives": int(nprim), "ms": float(np.mean(ms_env)),
                       "samples_per_s": nsamp / (float(np.mean(ms_env)) * 1e-3),
                       "max_distance_over_diagonal": float(dd.max()), "mean_distance_over_diagonal": float(dd.mean())}
    return out


def run_reference(args, w):
    """The reference arm: the CPU oracle (brute force, FP64 + exact predicates)
    as it stands on the host cores, each step a seeded tet sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    per_step = CPU_SAMPLES.get(args.config, CPU_SAMPLES["block_c2"])["ref"]
    times = []
    pieces = 0
    cores = 0
    for s in range(args.warmup + args.steps):
        sub = _sample(w.nt, per_step, 1000 + s)
        t0 = time.perf_counter()
        o = oracle.run(w, subset=sub)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pieces += len(o["tet"])
            cores = o["nthreads"]
    value = pieces / sum(times)
    sample = f"{per_step} of {w.nt} seeded tets per step ({100.0 * per_step / w.nt:.3g}%), all {w.ns} spheres"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[args.config], "precision": "fp64 + exact predicates",
                       "tets_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="blob_c3", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"])
    ap.add_argument("--k", type=int, default=None, help="power neighbours kept per mesh vertex")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling)")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precision (profiling)")
    ap.add_argument("--no-medial", action="store_true", help="skip the medial-mesh and envelope leg")
    ap.add_argument("--repair-shapes", type=int, default=64,
                    help="genus 0-5 slabs of the repair leg (0 skips it)")
    ap.add_argument("--batch-shapes", type=int, default=64,
                    help="shapes of the batching leg (0 skips it; the full batching workload has 256)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    w = make_workload(args.config)
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist
    from paper_2403_18761_gb300 import rpd_build, rpd_launch_count
    from paper_2403_18761_gb300.rpd import rpd_stats

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precision = args.precision or w.precision
    stream = torch.cuda.Stream(device=dev)

    V = torch.as_tensor(w.verts, dtype=torch.float64, device=dev)
    T = torch.as_tensor(w.tets, dtype=torch.int32, device=dev)
    C = torch.as_tensor(w.centers, dtype=torch.float64, device=dev)
    R = torch.as_tensor(w.radii, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    kk = args.k or w.k

    def step(Vd, Td, Cd, Rd):
        ctx = rpd_build(Vd, Td, Cd, Rd, precision=precision, k=kk, grid_bits=w.grid_bits, stream=stream)
        outs = []
        for kind in (1, 2, 3, 4):
            outs.append(ctx.rpd_euler(kind))
            outs.append(ctx.rpd_components(kind))
            outs.append(ctx.rpd_contractible(kind))
        return ctx, outs

    # ---- CUDA-core peaks of this GPU (the roofline denominators), measured
    # by the library's FMA-chain microbenchmark before the timed steps
    with torch.cuda.stream(stream):
        with ClockSampler(local) as pclk:
            peaks = fma_peaks()
    peaks["clocks"] = pclk.summary()
    mp = measured_peaks()
    peaks["hbm_gbs"] = mp.get("hbm_gbs")
    peaks["hbm_source"] = "MEASURED_PEAKS.json hbm_gbs (STREAM-style copy, of measured)" if mp.get("hbm_gbs") else None

    # ---- device-resident timing
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx, _ = step(V, T, C, R)
            ctx.rpd_destroy()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms, stage, pieces = [], [], 0
        launches0 = rpd_launch_count()
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx, outs = step(V, T, C, R)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                st = ctx.rpd_stats_get()
                stage.append(st)
                pieces += st["n_pieces"]
                ctx.rpd_destroy()
        torch.cuda.synchronize()
    launches = rpd_launch_count() - launches0
    clocks = clk.summary()
    t_step = max(ms)
    total_ms, value = job_throughput(sum(ms), pieces, world, dev)

    # ---- end to end through the C-ABI from pinned host buffers
    hV = torch.as_tensor(w.verts, dtype=torch.float64).pin_memory()
    hT = torch.as_tensor(w.tets, dtype=torch.int32).pin_memory()
    hC = torch.as_tensor(w.centers, dtype=torch.float64).pin_memory()
    hR = torch.as_tensor(w.radii, dtype=torch.float64).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in (hV, hT, hC, hR))
    e2e_ms, d2h, npieces = [], 0, 0
    with torch.cuda.stream(stream):
        for s in range(0 if args.no_e2e else args.warmup + args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Vd, Td, Cd, Rd = (x.to(dev, non_blocking=True) for x in (hV, hT, hC, hR))
            ctx, outs = step(Vd, Td, Cd, Rd)
            host, nbytes = ctx.tables_host()   # every table in one copy of the export buffer
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                e2e_ms.append(dt * 1e3)
                d2h = nbytes
                npieces = ctx.rpd_stats_get()["n_pieces"]
            ctx.rpd_destroy()
    e2e_value = npieces * len(e2e_ms) / (sum(e2e_ms) / 1e3) * world if e2e_ms else None

    st_mean = {k: float(np.mean([s[k] for s in stage]))
               for k in ("ms_prep", "ms_knn", "ms_cand", "ms_clip", "ms_clip_kernels", "ms_clip_span")}
    st_mean["ms_finalize"] = [float(np.mean([s["ms_finalize"][k] for s in stage])) for k in range(4)]
    last = stage[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config], "precision": precision, "tets": int(w.nt),
                   "spheres": int(w.ns), "pieces_per_step": int(last["n_pieces"]),
                   "l2": "256 MB buffer written between timed steps", "parallelism": "replicas"},
        "stages_ms": st_mean,
        "predicates": {"fast": last["pred_fast"], "fp64": last["pred_fp64"], "exact": last["pred_exact"],
                       "vertices_constructed": last["clip_vertices"]},
        "pairs": {"total": last["n_pairs"], "by_bin": last["bin_pairs"], "cut_by_bin": last["bin_cut"],
                  "whole_tets": last["whole_tets"], "cand_fallback": last["cand_fallback"], "k": kk},
        "elements": {"records": last["n_records"], "keys": last["n_keys"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps,
        "step_ms_max": t_step,
        "peaks": peaks,
    }
    # ---- the other precision, same step (FP32-filtered vs FP64 throughput)
    ostage = []
    if not args.no_compare:
        other = "fp64" if precision == "fp32" else "fp32"
        oms = []
        with torch.cuda.stream(stream):
            for it in range(args.warmup + args.steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx = rpd_build(V, T, C, R, precision=other, k=kk, grid_bits=w.grid_bits, stream=stream)
                for kind in (1, 2, 3, 4):
                    ctx.rpd_euler(kind), ctx.rpd_components(kind), ctx.rpd_contractible(kind)
                e1.record(stream)
                e1.synchronize()
                st = ctx.rpd_stats_get()
                if it >= args.warmup:
                    oms.append(e0.elapsed_time(e1))
                    ostage.append(st)
                npo = st["n_pieces"]
                ctx.rpd_destroy()
        ovalue = npo * len(oms) / (sum(oms) / 1e3)
        v32, v64 = (value, ovalue) if precision == "fp32" else (ovalue, value)
        line["precision_compare"] = {"fp32": v32, "fp64": v64, "fp32_over_fp64": v32 / v64, "unit": UNIT,
                                     "pieces_equal": bool(npo == last["n_pieces"]),
                                     "ms_clip_kernels": {precision: st_mean["ms_clip_kernels"],
                                                         other: float(np.mean([q["ms_clip_kernels"] for q in ostage]))}}
    stage64 = ostage if precision == "fp32" else stage
    line["roofline"] = clip_roofline(stage, kk, args.config, precision, peaks, peaks["hbm_gbs"],
                                     stage64=stage64 if stage64 else None)
    # the legs below are reported by rank 0 alone, so only rank 0 runs them
    if args.batch_shapes > 0 and rank == 0:
        try:
            line["batch"] = batch_leg(args.batch_shapes, args.steps, args.warmup, stream, flush, dev)
        except Exception as e:   # reported in the line; the headline stands on its own
            line["batch"] = {"shapes": args.batch_shapes, "error": f"{type(e).__name__}: {e}"}
    if not args.no_medial and rank == 0:
        try:
            line.update(medial_envelope_leg(w, precision, kk, stream, dev))
        except Exception as e:
            line["medial"] = {"error": f"{type(e).__name__}: {e}"}
    if args.repair_shapes > 0 and rank == 0:
        try:
            line["repair"] = repair_leg(args.repair_shapes, stream, dev)
        except Exception as e:
            line["repair"] = {"shapes": args.repair_shapes, "error": f"{type(e).__name__}: {e}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, legs, (sub, o) = cpu_baselines(w, args.config)
        line["cpu_baseline"] = cb
        line["cpu_legs"] = legs
        errs = {}
        for prec in ("fp32", "fp64"):
            with torch.cuda.stream(stream):
                ctx = rpd_build(V, T, C, R, precision=prec, k=kk, grid_bits=w.grid_bits, stream=stream)
                pieces = [x.cpu().numpy() for x in ctx.rpd_pieces()]
                ctx.rpd_destroy()
            errs[prec] = volume_error(w, pieces, sub, o)
        line["error_vs_oracle"] = errs[precision]
        line["error_vs_oracle_by_precision"] = errs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
