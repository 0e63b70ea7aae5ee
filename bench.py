"""Benchmark: restricted (tet, sphere) pieces per second, including the
fractional Euler characteristic, connected components and contractibility of
every RPC/RPF/RPE/RPV, on one GB300.

One step = rpd_build + rpd_euler/rpd_components/rpd_contractible for every
element kind (all of the hot path) on the genus-3 block workload (4x2x1 box
with three through-holes, ~200k tets, 2k near-medial spheres, FP32-filtered
clipping with FP64/exact fallback, k = 32).  Inputs are seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config block_c2|torus_c1|blob_c3] [--precision fp32|fp64]
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


# Algorithmic FP32 work of the clip stage (Tet-Cell clipping, Sec. 5.2):
# one filtered sign test F.C of a live polytope vertex against a new radical
# plane is 3 FMA + 1 MUL = 7 flop (its error bound is stored with the vertex).
# A vertex constructed on a new plane takes the cofactors of its m radical-plane
# rows (m = 1: a selection, 0 flop; m = 2: three 2x2 minors, 9 flop; m = 3:
# four 3x3 cofactors, 56 flop) plus its orientation test and stored bound
# (17 flop).
FLOP_SIGN_TEST = 7
FLOP_NEW_VERTEX = (17, 26, 73)   # by m = 1, 2, 3
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of the clip kernels of one step (k_clip over all
# bins + k_whole) on block_c2, from one ncu capture of the current kernels
# (profiles/clip_block_c2.md); None once the kernels change.
CLIP_TRAFFIC_BYTES = {("block_c2", "fp32"): 67.86e6}


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


def clip_roofline(stage, n_sm, workload, precision):
    """FP32 ALU roofline of the clip kernels, from the counters of the timed
    steps and the clip-kernel span timed by the library's CUDA events on the
    launching streams."""
    peaks = measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    flop, ms = [], []
    for s in stage:
        tests = s["pred_fast"] + s["pred_fp64"] + s["pred_exact"]
        nv = s["clip_vertices"]
        flop.append(FLOP_SIGN_TEST * max(tests - sum(nv), 0) + sum(f * n for f, n in zip(FLOP_NEW_VERTEX, nv)))
        ms.append(s["ms_clip_kernels"])
    achieved = float(np.mean(flop)) / (float(np.mean(ms)) * 1e-3) / 1e12
    return {"kernel": "k_clip over all candidate-count bins + k_whole (side by side on the bin streams; "
                      "timed to the end of the record kernels that follow them there)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": CLIP_TRAFFIC_BYTES.get((workload, precision)), "flop_per_launch": float(np.mean(flop)),
            "ms_per_launch": float(np.mean(ms)),
            "peak_source": f"derived FP32: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {mhz:.0f} MHz "
                           "(sm_max_mhz of MEASURED_PEAKS.json)"}


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


def oracle_baseline(w, frac, seed=20240318, nthreads=None):
    """Time the oracle (as it stands) on a seeded tet sample of the workload."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    n = max(1, int(round(frac * w.nt)))
    sub = np.sort(rng.choice(w.nt, size=n, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    o = oracle.run(w, subset=sub, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return dict(value=len(o["tet"]) / dt, unit=UNIT, cores=o["nthreads"], kind="oracle",
                sample=f"{n} of {w.nt} tets ({100 * frac:.1f}%, seed {seed}), all {w.ns} spheres, "
                       f"brute-force C oracle; {len(o['tet'])} pieces in {dt:.2f} s"), (sub, o)


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


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    frac = args.ref_frac
    times = []
    pieces = 0
    for s in range(args.warmup + args.steps):
        import oracle
        rng = np.random.default_rng(1000 + s)
        sub = np.sort(rng.choice(w.nt, size=max(1, int(frac * w.nt)), replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        o = oracle.run(w, subset=sub)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pieces += len(o["tet"])
            cores = o["nthreads"]
    value = pieces / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[args.config], "precision": "fp64 + exact predicates",
                       "sample_fraction": frac},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{frac * 100:.1f}% seeded tet sample per step, all spheres"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="block_c2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"])
    ap.add_argument("--k", type=int, default=None, help="power neighbours kept per mesh vertex")
    ap.add_argument("--cpu-frac", type=float, default=0.05)
    ap.add_argument("--ref-frac", type=float, default=0.01)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling)")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precision (profiling)")
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
        "roofline": clip_roofline(stage, torch.cuda.get_device_properties(dev).multi_processor_count, args.config,
                                  precision),
        "step_ms_max": t_step,
    }
    # ---- the other precision, same step (FP32-filtered vs FP64 throughput)
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
                if it >= args.warmup:
                    oms.append(e0.elapsed_time(e1))
                npo = ctx.rpd_stats_get()["n_pieces"]
                ctx.rpd_destroy()
        ovalue = npo * len(oms) / (sum(oms) / 1e3)
        v32, v64 = (value, ovalue) if precision == "fp32" else (ovalue, value)
        line["precision_compare"] = {"fp32": v32, "fp64": v64, "fp32_over_fp64": v32 / v64, "unit": UNIT,
                                     "pieces_equal": bool(npo == last["n_pieces"])}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, (sub, o) = oracle_baseline(w, args.cpu_frac)
        line["cpu_baseline"] = cb
        with torch.cuda.stream(stream):
            ctx = rpd_build(V, T, C, R, precision=precision, k=kk, grid_bits=w.grid_bits, stream=stream)
            pieces = [x.cpu().numpy() for x in ctx.rpd_pieces()]
            ctx.rpd_destroy()
        line["error_vs_oracle"] = volume_error(w, pieces, sub, o)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
