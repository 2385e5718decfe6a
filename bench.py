#!/usr/bin/env python
"""Benchmark: forward + back projection on the jittered Kuhn 96^3 workload,
with the batched workload (24 problems of uneven size, 4 channels, one
persistent launch per direction under a CUDA graph) nested in the same line.

One step = tetproj_forward (b = A mu) followed by tetproj_backward of that
projection (x = A^T b): 512 x 512 x 360 = 94,371,840 cone-beam rays through
5,308,416 tets, each way.  `value` is rays/s of such fwd+back pairs on the
device (inputs resident in HBM); `e2e` is the same through the C ABI with host
buffers (pinned H2D of mu, D2H of the projection and the backprojection every
step).  The filtered FP32 path is the product; the plain FP64 path is timed
beside it for the ratio, with its FP64-ALU roofline.  `batched` times the
24-problem workload the same way (--no-batched leaves it out).  Under
torchrun every rank runs an independent replica (the operator shards over
rays with no exchange in the forward; this build has no cross-GPU step), so
value = all ranks' rays / max time.

Other workloads (--workload): kuhn8 (the tiny plain-method case), cubic64 (the
robustness case, with its 1M adversarial rays timed separately), recon64 (the
differentiation case: ms per Adam iteration through the autograd wrapper),
batch24 / batch6s (the batched workload alone), c5pK (problem K of the
batched workload alone, one channel), kuhn24 / kuhn64 / kuhn64s / kuhn96s
(smaller copies for profiling).

--impl reference times the CPU oracle on a bounded sample of the same rays, on
the host cores: the oracle walker by default (FP64 clipping of the tets each
ray crosses), the brute-force clipper with --cpu-oracle clipper.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+back projection rays/s & Gsegments/s vs plain FP64 GPU path, 1×GB300"
HBM_FALLBACK = 6800.0
# Algorithmic bytes per walk step (segment), filtered FP32 path: the records
# one step must fetch in an SoA layout -- vertex ids 16 + adjacency 16 + the
# one new FP32 vertex 12 + mu 4C (forward) or an FP32 read-modify-write 4C+4C
# (backward): 48 / 60 B forward and 52 / 76 B backward for C = 1 / 4.  Per ray
# add 4C bytes of projection, and the BVH boxes / boundary faces visited.
BYTES_STEP = {("fwd", 1): 48, ("fwd", 4): 60, ("bwd", 1): 52, ("bwd", 4): 76}
BYTES_RAY = lambda C: 4 * C          # proj written (fwd) or read (bwd)
BYTES_BOX = 32                       # one BVH child box (half of a 64-byte node)
BYTES_FACE = 48                      # one boundary face record
# what this layout actually moves per step: one 64-byte record + mu / RMW
LAYOUT_STEP = {("fwd", 1): 68, ("fwd", 4): 80, ("bwd", 1): 72, ("bwd", 4): 96}
# ... and with the FP64 accumulator of the default C = 1 backprojection: one
# 64-byte record + an 8-byte read-modify-write of the accumulator (red.f64)
LAYOUT_STEP_ACC64 = 80


PROFILES = os.path.join(ROOT, "profiles")
# DRAM bytes per segment of the filtered walk kernels, from an ncu capture of
# a smaller launch of the same mesh (profiles/walk32_kuhn96s_traffic.md), and
# FP64 operations per segment of the plain walk (profiles/walk64_kuhn64s_fp64.md);
# both are used only while the walk sources hash to the value recorded there.
TRAFFIC_FILE = os.path.join(PROFILES, "walk32_kuhn96s_traffic.md")
PROFILED_TILE = "16x8"  # the launch configuration of that capture (default options)
FP64OPS_FILE = os.path.join(PROFILES, "walk64_kuhn64s_fp64.md")
WALK_SOURCES = ["kernels.cu", "kernels.cuh", "predicates.cuh", "tetproj_internal.h"]


def walk_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in WALK_SOURCES:
        with open(os.path.join(ROOT, "paper_1908_06909_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_per_segment(path, key):
    """{fwd, bwd} per-segment figures recorded under `key` in a committed
    profile summary, or None if the walk sources changed since the capture."""
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        parts = line.split()
        if len(parts) == 2 and parts[0] == "source_sha256":
            vals["sha"] = parts[1]
        if parts and parts[0] == key:
            vals["v"] = {k: float(v) for k, v in (q.split("=") for q in parts[1:])}
    if vals.get("sha") != walk_sources_sha() or "v" not in vals:
        return None
    return vals["v"]


def max_over_ranks(ms, dist, device="cuda"):
    """The slowest rank's time (every rank gets it); the value itself without
    a process group."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, ms):
    """Whole-job rate: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms while the timed region runs."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def build_workload(args):
    import workloads as W
    if args.workload == "kuhn96":
        return W.config2()
    if args.workload == "kuhn24":   # small case for quick runs
        return W.config2(n_cells=24, det=128, pitch=0.05, nangles=32)
    if args.workload == "kuhn64":   # 1.57M tets, 256^2 x 180 (11.8M rays)
        return W.config2(n_cells=64, det=256, pitch=0.025, nangles=180)
    if args.workload == "kuhn64s":  # same mesh, 30 angles: profiler-sized launches
        return W.config2(n_cells=64, det=256, pitch=0.025, nangles=30)
    raise SystemExit(f"unknown workload {args.workload}")


L2_BYTES = 129e6


def l2_note(nt, nrays, C):
    rec, proj = nt * 64, nrays * 4 * C
    kind = "larger" if rec + proj > L2_BYTES else "SMALLER"
    return (f"inputs {kind} than L2, not flushed (tet records {rec / 1e6:.0f} MB, "
            f"projections {proj / 1e6:.0f} MB)")


CPU_SAMPLE = {"walker": 20000, "clipper": 256}


def cpu_baseline(w, nsample, threads=None, kind="walker"):
    """The oracle as it stands, on `nsample` rays spread over the workload:
    forward (b_j for the sampled rays) and backward (A^T y restricted to
    those rays); returns fwd+back ray pairs per second.  kind "walker": the
    oracle walker (each a_ij from the clipper, only for the tets the ray
    crosses, found over the oracle's own adjacency; rays with near-ties over
    all tets), its adjacency built outside the timed region; "clipper": the
    brute-force clipper (every ray against every tet)."""
    import oracle
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(w.geom.nrays, nsample, replace=False))
    y = rng.uniform(size=nsample)
    threads = threads or oracle.default_threads()
    mu = np.asarray(w.mu)
    if kind == "walker":
        wk = oracle.Walker(w.verts, w.tets)
        t0 = time.perf_counter()
        wk.forward_cone(mu, w.geom, idx, threads=threads)
        wk.backward_cone(y, w.geom, idx, threads=threads)
        dt = time.perf_counter() - t0
    else:
        S, P = oracle.cone_rays(w.geom, idx)
        t0 = time.perf_counter()
        oracle.forward_rays(w.verts, w.tets, mu, S, P, threads=threads)
        oracle.backward_rays(w.verts, w.tets, y, S, P, threads=threads)
        dt = time.perf_counter() - t0
    return nsample / dt, threads, dt, idx.size


def cpu_sample_text(kind, n, nrays):
    if kind == "walker":
        return (f"{n} of {nrays} rays per step (fwd + back), oracle walker: FP64 clipping of the "
                f"tets each ray crosses, found over the oracle's own adjacency")
    return f"{n} of {nrays} rays per step (fwd + back), brute-force FP64 clipping over all tets"


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = build_workload(args)
    kind = args.cpu_oracle
    n = args.cpu_sample or CPU_SAMPLE[kind]
    for _ in range(args.warmup):
        cpu_baseline(w, max(8, n // 16), kind=kind)
    times = []
    for _ in range(args.steps):
        v, cores, dt, ns = cpu_baseline(w, n, kind=kind)
        times.append(dt)
    value = n / float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "nt": int(w.tets.shape[0]),
                   "rays_per_step": n, "note": "bounded ray sample of the same workload"},
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                         "sample": cpu_sample_text(kind, n, w.geom.nrays)},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_workload(name):
    """The batched workload: 24 problems (config-5 sizes), or a reduced copy."""
    import workloads as W
    if name == "batch24":
        specs = W.config5_specs()
    elif name == "batch6s":  # small case for quick runs
        specs = [(3, 16, 5), (8, 48, 9), (5, 24, 3), (12, 40, 7), (4, 32, 12), (6, 20, 4)]
    elif name == "batch1k64":  # one problem, profiler-sized (jittered Kuhn 64^3, 256^2 x 30)
        specs = [(64, 256, 30)]
    else:
        raise SystemExit(f"unknown workload {name}")
    return [W.config5_problem(k, n, N, na, channels=4) for k, (n, N, na) in enumerate(specs)]


def run_batch(args, tp, torch, dist, rank, world, local):
    """All problems forward + backward, 4 channels, filtered FP32, as one
    persistent work-queue launch per direction replayed from CUDA graphs;
    tiles, ordering and scatter from the autotuner.  Beside it: the same
    problems as sequential single-problem calls (same options), and the plain
    FP64 path on every 8th angle of each problem, scaled by ray count."""
    from paper_1908_06909_gb300 import autotune as A
    C = 4
    t_build = time.perf_counter()
    ws = batch_workload(args.workload)
    meshes = [tp.Mesh(w.verts, w.tets) for w in ws]
    geos = [tp.Geometry.from_cone(w.geom) for w in ws]
    t_build = time.perf_counter() - t_build
    t_tune = time.perf_counter()
    cache = A.Cache(args.tune_cache, device=torch.cuda.get_device_name(), version=tp.version())
    if args.no_tune:  # fixed tiles from --tile / --scatter, Morton order
        tu, tv = (int(x) for x in args.tile.split("x"))
        sc = tp.SCATTER_WARP if args.scatter == "warp" else tp.SCATTER_ATOMIC
        tiles = [(tu, tv, tp.ORDER_MORTON, sc)] * len(ws)
    else:
        choices = A.tune_batch(tp, meshes, geos, channels=C, cache=cache, reps=2)
        tiles = [c.row() for c in choices]
    t_tune = time.perf_counter() - t_tune
    b = tp.Batch(meshes, geos, channels=C, tiles=tiles)
    for k, w in enumerate(ws):
        b.mu[k].copy_(torch.tensor(w.mu, dtype=torch.float32))
    stream = torch.cuda.current_stream()
    nrays = b.nrays

    # work counts per direction (one untimed pass each, outside the graphs)
    for m in meshes:
        m.stats_reset()
    b.forward()
    sf = _sum_stats([m.stats() for m in meshes])
    for k in range(b.n):
        b.y[k].copy_(b.proj[k])
    for m in meshes:
        m.stats_reset()
    b.backward()
    sb = _sum_stats([m.stats() for m in meshes])
    assert sf["error"] == 0 and sb["error"] == 0, (sf, sb)
    torch.cuda.synchronize()
    gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    launches0 = tp.launch_count()
    with torch.cuda.graph(gf):
        b.forward()
    with torch.cuda.graph(gb):
        b.backward()
    launches_per_step = tp.launch_count() - launches0  # kernels in the two graphs
    for _ in range(args.warmup):
        gf.replay()
        gb.replay()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for k in range(args.steps):
            evs[k][0].record(stream)
            gf.replay()
            evs[k][1].record(stream)
            gb.replay()
            evs[k][2].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_step = max_over_ranks(start.elapsed_time(end), dist) / args.steps
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    bwd_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    value = job_throughput(world, nrays, ms_step)
    segs = sf["segments"] + sb["segments"]

    # the same problems as sequential single-problem calls (same options)
    opts = [tp.make_options(channels=C, tile=(r[0], r[1]), order=r[2], scatter=r[3])
            for r in tiles]
    def singles():
        for k in range(b.n):
            tp.forward(meshes[k], geos[k], b.mu[k], out=b.proj[k], options=opts[k])
            tp.backward(meshes[k], geos[k], b.y[k], out=b.mu_out[k], options=opts[k])
    singles()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    singles()
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1)

    # plain FP64 and filtered single calls on every 8th angle, scaled by rays
    plain_ms = filt_ms = 0.0
    rel_num = rel_den = 0.0
    for k, w in enumerate(ws):
        sel = w.geom.angles[::8]
        gs = tp.Geometry(w.geom.dso, w.geom.dsd, w.geom.nu, w.geom.nv, w.geom.du, w.geom.dv, sel)
        mu64 = b.mu[k].double()
        o64 = tp.make_options(precision=tp.PLAIN_FP64, channels=C, tile=(tiles[k][0], tiles[k][1]),
                              order=tiles[k][2], scatter=tiles[k][3])
        p64 = tp.forward(meshes[k], gs, mu64, options=o64)
        x64 = tp.backward(meshes[k], gs, p64, options=o64)
        p32 = tp.forward(meshes[k], gs, b.mu[k], options=opts[k])
        x32 = tp.backward(meshes[k], gs, p32, options=opts[k])
        torch.cuda.synchronize()
        for prec, fn in (("f64", lambda: (tp.forward(meshes[k], gs, mu64, out=p64, options=o64),
                                          tp.backward(meshes[k], gs, p64, out=x64, options=o64))),
                         ("f32", lambda: (tp.forward(meshes[k], gs, b.mu[k], out=p32, options=opts[k]),
                                          tp.backward(meshes[k], gs, p32, out=x32, options=opts[k])))):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn()
            a1.record(stream)
            torch.cuda.synchronize()
            scaled = a0.elapsed_time(a1) * geos[k].nrays / gs.nrays
            if prec == "f64":
                plain_ms += scaled
            else:
                filt_ms += scaled
        rel_num += float((p32.double() - p64).abs().sum())
        rel_den += float(p64.abs().sum())
        del p64, x64, p32, x32, mu64

    # end to end with host buffers: H2D of every mu, D2H of every projection
    # and backprojection (the graphs read and write the bound tensors).  The
    # copies run on a second stream beside the walks: the projections' D2H
    # and the next step's H2D during the backprojection, the backprojections'
    # D2H during the next forward projection; events keep every buffer's
    # writer after its previous copy.
    mu_h = [torch.empty_like(x, device="cpu").pin_memory() for x in b.mu]
    for k in range(b.n):
        mu_h[k].copy_(b.mu[k])
    proj_h = [torch.empty_like(x, device="cpu").pin_memory() for x in b.proj]
    back_h = [torch.empty_like(x, device="cpu").pin_memory() for x in b.mu_out]
    cs = torch.cuda.Stream()
    ev_f, ev_b, ev_c1, ev_c2 = (torch.cuda.Event() for _ in range(4))
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(b.n):
        b.mu[k].copy_(mu_h[k], non_blocking=True)
    for step in range(args.steps):
        if step > 0:
            stream.wait_event(ev_c1)  # next mu in, previous projections out
        gf.replay()
        ev_f.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_f)
            for k in range(b.n):
                proj_h[k].copy_(b.proj[k], non_blocking=True)
            if step + 1 < args.steps:
                for k in range(b.n):
                    b.mu[k].copy_(mu_h[k], non_blocking=True)
            ev_c1.record(cs)
        for k in range(b.n):
            b.y[k].copy_(b.proj[k])
        if step > 0:
            stream.wait_event(ev_c2)  # previous backprojections out
        gb.replay()
        ev_b.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_b)
            for k in range(b.n):
                back_h[k].copy_(b.mu_out[k], non_blocking=True)
            ev_c2.record(cs)
    stream.wait_event(ev_c1)
    stream.wait_event(ev_c2)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    h2d = sum(x.numel() * 4 for x in mu_h)
    d2h = sum(x.numel() * 4 for x in proj_h) + sum(x.numel() * 4 for x in back_h)
    del mu_h, proj_h, back_h

    hbm, peak_kind = peaks()
    def alg_bytes(s, kind, table=BYTES_STEP):
        return (s["segments"] * table[(kind, C)] + s["rays"] * BYTES_RAY(C) +
                s["bvh_nodes"] * BYTES_BOX + s["bvh_faces"] * BYTES_FACE)
    dom = "bwd" if bwd_ms >= fwd_ms else "fwd"
    dom_ms = bwd_ms if dom == "bwd" else fwd_ms
    dom_bytes = alg_bytes(sb if dom == "bwd" else sf, dom)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": f"k_batch32<4,{'MODE_BWD' if dom == 'bwd' else 'MODE_FWD'}>",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "peak_kind": peak_kind, "bytes_per_launch": dom_bytes,
            "ms_per_launch": dom_ms, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
            "layout_gbs": alg_bytes(sb if dom == "bwd" else sf, dom, LAYOUT_STEP) / (dom_ms / 1e3) / 1e9}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        kind = args.cpu_oracle
        per = max(1, (args.cpu_sample or CPU_SAMPLE[kind]) // len(ws))
        dt = 0.0
        n_cpu = 0
        for w in ws:
            rng = np.random.default_rng(777)
            idx = np.sort(rng.choice(w.geom.nrays, per, replace=False))
            yv = rng.uniform(size=(per, C))
            if kind == "walker":
                wk = oracle.Walker(w.verts, w.tets)  # adjacency built outside the timing
                t0 = time.perf_counter()
                wk.forward_cone(w.mu, w.geom, idx)
                wk.backward_cone(yv, w.geom, idx)
            else:
                S, P = oracle.cone_rays(w.geom, idx)
                t0 = time.perf_counter()
                oracle.forward_rays(w.verts, w.tets, w.mu, S, P)
                oracle.backward_rays(w.verts, w.tets, yv, S, P)
            dt += time.perf_counter() - t0
            n_cpu += per
        how = ("oracle walker" if kind == "walker" else "brute-force FP64 clipping")
        cpu = {"value": n_cpu / dt, "unit": "rays/s", "cores": oracle.default_threads(),
               "kind": "oracle", "sample": f"{per} rays of each of {len(ws)} problems (fwd + back, "
                                           f"4 channels), {how}, {dt:.1f} s"}
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "problems": len(ws),
                       "nt_total": int(sum(m.nt for m in meshes)), "rays_per_step": nrays,
                       "channels": C, "precision": "filtered", "launch": "persistent work queue, CUDA graph",
                       "work_item": "32-ray warp slice of a tile", "tiles": tiles,
                       "l2": "inputs larger than L2", "parallelism": f"replicas{world}"},
            "gsegments_per_s": job_throughput(world, segs, ms_step) / 1e9,
            "segments_per_step": segs,
            "unbatched": {"ms_per_step": single_ms, "value": nrays / (single_ms / 1e3),
                          "speedup_batched": single_ms / ms_step},
            "plain_fp64": {"ms_per_step_est": plain_ms, "value": nrays / (plain_ms / 1e3),
                           "filtered_single_ms_est": filt_ms,
                           "speedup_batched_vs_plain": plain_ms / ms_step,
                           "filtered_vs_plain_rel_l1_diff": rel_num / max(rel_den, 1e-300),
                           "sample": "every 8th angle of each problem, time scaled by ray count"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": job_throughput(world, nrays, e2e_ms), "unit": "rays/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            # kernels captured in the two graphs (counted by the library at
            # capture) times the replays of the timed region
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clk.summary(),
            "host_s": {"build": t_build, "tune": t_tune},
            "stats": {"fwd": sf, "bwd": sb},
        }
    b.close()
    del b, meshes, geos
    torch.cuda.empty_cache()
    return line


def _sum_stats(rows):
    out = {}
    for r in rows:
        for k, v in r.items():
            out[k] = out.get(k, 0) + v
    return out


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kuhn96")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="rays of the CPU oracle sample (0: 20000 for the walker, 256 for the clipper)")
    ap.add_argument("--cpu-oracle", default="walker", choices=["walker", "clipper"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: leave out the nested batched measurement")
    ap.add_argument("--batched-workload", default="batch24")
    ap.add_argument("--scatter", default="atomic", choices=["atomic", "warp", "sort"])
    ap.add_argument("--tile", default="16x8")
    ap.add_argument("--tune-cache", default=None)
    ap.add_argument("--acc", default="auto", choices=["auto", "f32", "f64"],
                    help="accumulator of the filtered backprojection (auto: FP64 at C = 1)")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workloads: fixed --tile/--scatter instead of the autotuner")
    return ap.parse_args(argv)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import __graft_entry__ as g
    g.build_library()
    import paper_1908_06909_gb300 as tp

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.workload.startswith("batch"):
        line = run_batch(args, tp, torch, dist, rank, world, local)
    elif args.workload == "recon64":
        line = run_recon(args, tp, torch, dist, rank, world, local)
    else:
        line = run_single(args, tp, torch, dist, rank, world, local)
        if args.workload == "kuhn96" and not args.no_batched:
            # the batched workload, timed the same way, nested in the same line
            bargs = parse_args([])
            bargs.workload = args.batched_workload
            bargs.steps = max(3, min(args.steps, 5))
            bargs.warmup = 3
            bargs.no_cpu = True
            bargs.tune_cache = args.tune_cache
            bl = run_batch(bargs, tp, torch, dist, rank, world, local)
            if bl is not None:
                keep = ["value", "unit", "ms_per_step", "steps", "warmup", "config",
                        "gsegments_per_s", "segments_per_step", "unbatched", "plain_fp64",
                        "roofline", "e2e", "gpu_launches", "clocks", "host_s"]
                line["batched"] = {k: bl[k] for k in keep if k in bl}
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def build_single_workload(args):
    import workloads as W
    if args.workload == "kuhn8":       # the tiny plain-method case (8^3 Kuhn, 64^2 x 32)
        return W.config1()
    if args.workload == "cubic64":     # the robustness case (detector rays; adversarial below)
        return W.config3()
    if args.workload == "kuhn96s":     # the bench mesh, 8 angles: profiler-sized launches
        return W.config2(nangles=8)
    if args.workload.startswith("c5p"):  # one problem of the batched workload, one channel
        k = int(args.workload[3:])
        n, N, na = W.config5_specs()[k]
        w = W.config5_problem(k, n, N, na, channels=1)
        w.mu = w.mu[:, 0].copy()
        return w
    return build_workload(args)


def run_single(args, tp, torch, dist, rank, world, local):
    """One problem: forward + backward per step, filtered FP32 (the product),
    the plain FP64 path beside it, e2e with host buffers, roofline, oracle."""
    w = build_single_workload(args)
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    tu, tv = (int(x) for x in args.tile.split("x"))
    opt = tp.make_options(tile=(tu, tv), scatter={"atomic": tp.SCATTER_ATOMIC,
                                                  "warp": tp.SCATTER_WARP,
                                                  "sort": tp.SCATTER_SORT}[args.scatter],
                          flags={"auto": 0, "f64": tp.FLAG_ACC64, "f32": tp.FLAG_ACC32}[args.acc])
    acc = ("f32" if args.scatter == "sort" else "f64") if args.acc == "auto" else args.acc
    C = 1
    mu = torch.tensor(w.mu, dtype=torch.float32, device="cuda")
    proj = torch.empty(geo.shape, dtype=torch.float32, device="cuda")
    back = torch.empty(mesh.nt, dtype=torch.float32, device="cuda")
    mesh.reserve(tp.FILTERED, 1)
    stream = torch.cuda.current_stream()

    def step():
        tp.forward(mesh, geo, mu, out=proj, options=opt)
        tp.backward(mesh, geo, proj, out=back, options=opt)

    # per-direction work counts (one untimed pass each)
    mesh.stats_reset()
    tp.forward(mesh, geo, mu, out=proj, options=opt)
    sf = mesh.stats()
    mesh.stats_reset()
    tp.backward(mesh, geo, proj, out=back, options=opt)
    sb = mesh.stats()
    assert sf["error"] == 0 and sb["error"] == 0, (sf, sb)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = tp.launch_count()
    with ClockSampler(local) as clk:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for k in range(args.steps):
            e0, e1, e2 = evs[k]
            e0.record(stream)
            tp.forward(mesh, geo, mu, out=proj, options=opt)
            e1.record(stream)
            tp.backward(mesh, geo, proj, out=back, options=opt)
            e2.record(stream)
        end.record(stream)
        torch.cuda.synchronize()
    launches = tp.launch_count() - launches0
    if dist:
        dist.barrier()
    total_ms = start.elapsed_time(end)
    fwd_ms = float(np.mean([a.elapsed_time(b) for a, b, _ in evs]))
    bwd_ms = float(np.mean([b.elapsed_time(c) for _, b, c in evs]))
    ms_step = max_over_ranks(total_ms, dist) / args.steps
    nrays = geo.nrays
    value = job_throughput(world, nrays, ms_step)
    segs = sf["segments"] + sb["segments"]

    # plain FP64 path (the ratio's denominator), same step, with its FP64-ALU
    # roofline: FP64 operations per segment (ncu capture) x segments over the
    # timed call, against the measured FP64 FMA rate
    plain = None
    if args.plain_steps > 0:
        mu64 = mu.double()
        proj64 = torch.empty(geo.shape, dtype=torch.float64, device="cuda")
        back64 = torch.empty(mesh.nt, dtype=torch.float64, device="cuda")
        o64 = tp.make_options(precision=tp.PLAIN_FP64, tile=(tu, tv), scatter=opt.scatter)
        mesh.stats_reset()
        tp.forward(mesh, geo, mu64, out=proj64, options=o64)
        sf64 = mesh.stats()
        mesh.stats_reset()
        tp.backward(mesh, geo, proj64, out=back64, options=o64)
        sb64 = mesh.stats()
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        pf = pb = 0.0
        for _ in range(args.plain_steps):
            a.record(stream)
            tp.forward(mesh, geo, mu64, out=proj64, options=o64)
            b.record(stream)
            tp.backward(mesh, geo, proj64, out=back64, options=o64)
            c.record(stream)
            torch.cuda.synchronize()
            pf += a.elapsed_time(b)
            pb += b.elapsed_time(c)
        pf /= args.plain_steps
        pb /= args.plain_steps
        pms = pf + pb
        rel = float(((proj.double() - proj64).abs().sum() / proj64.abs().sum()).item())
        fp64_peak = tp.fma64_peak_tflops()
        ops = profile_per_segment(FP64OPS_FILE, "fp64_ops_per_segment")
        pdom = "bwd" if pb >= pf else "fwd"
        pdom_ms = pb if pdom == "bwd" else pf
        proof = {"bound": "alu", "kernel": f"k_walk64<1,{'MODE_BWD' if pdom == 'bwd' else 'MODE_FWD'}>",
                 "peak": fp64_peak, "unit": "TFLOP/s", "peak_kind": "measured (FP64 FMA probe)",
                 "ms_per_launch": pdom_ms, "fwd_ms": pf, "bwd_ms": pb}
        if ops is not None:
            flops = ops[pdom] * (sb64 if pdom == "bwd" else sf64)["segments"]
            proof.update(achieved=flops / (pdom_ms / 1e3) / 1e12, frac=flops / (pdom_ms / 1e3) / 1e12 / fp64_peak,
                         flops_per_launch=flops, ops_per_segment=ops[pdom],
                         ops_note="FP64 operations per segment (2 per FMA) from profiles/walk64_kuhn64s_fp64.md")
        else:
            proof.update(achieved=None, frac=None, ops_note="no FP64 operation count for this build")
        plain = {"value": nrays / (pms / 1e3), "unit": "rays/s", "ms_per_step": pms,
                 "speedup_filtered_vs_plain": (nrays / (ms_step / 1e3)) / (nrays / (pms / 1e3)),
                 "filtered_vs_plain_rel_l1_diff": rel, "roofline": proof,
                 "segments": {"fwd": sf64["segments"], "bwd": sb64["segments"]}}
        del proj64, back64, mu64

    # end to end through the public API with host buffers
    mu_h = torch.empty(mesh.nt, dtype=torch.float32, pin_memory=True)
    mu_h.copy_(mu.cpu())
    proj_h = torch.empty(geo.shape, dtype=torch.float32, pin_memory=True)
    back_h = torch.empty(mesh.nt, dtype=torch.float32, pin_memory=True)
    # The copies run on a second stream beside the walks: the projection's D2H
    # and the next step's H2D (into the other of two input buffers) during the
    # backprojection, the backprojection's D2H during the next forward
    # projection; events keep every buffer's writer after its previous copy.
    mu_d = [torch.empty_like(mu), torch.empty_like(mu)]
    cs = torch.cuda.Stream()
    ev_f, ev_b, ev_c1, ev_c2 = (torch.cuda.Event() for _ in range(4))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    mu_d[0].copy_(mu_h, non_blocking=True)
    for step in range(args.steps):
        if step > 0:
            stream.wait_event(ev_c1)  # this step's mu in, previous projection out
        tp.forward(mesh, geo, mu_d[step % 2], out=proj, options=opt)
        ev_f.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_f)
            proj_h.copy_(proj, non_blocking=True)
            if step + 1 < args.steps:
                mu_d[(step + 1) % 2].copy_(mu_h, non_blocking=True)
            ev_c1.record(cs)
        if step > 0:
            stream.wait_event(ev_c2)  # previous backprojection out
        tp.backward(mesh, geo, proj, out=back, options=opt)
        ev_b.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_b)
            back_h.copy_(back, non_blocking=True)
            ev_c2.record(cs)
    stream.wait_event(ev_c1)
    stream.wait_event(ev_c2)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / args.steps
    e2e = {"value": job_throughput(world, nrays, max_over_ranks(e2e_ms, dist)), "unit": "rays/s",
           "h2d_bytes_per_step": mu_h.numel() * 4,
           "d2h_bytes_per_step": proj_h.numel() * 4 + back_h.numel() * 4}
    del mu_h, proj_h, back_h, mu_d

    # roofline of the dominant walk (events around each call; the O(nt)
    # permutation kernels inside the call are < 0.1% of it).  The default
    # backprojection at C = 1 reduces into an FP64 accumulator: the kernel is
    # k_walk32<1,MODE_BWD64>, and its layout moves 8-byte reductions.
    hbm, peak_kind = peaks()
    def alg_bytes(s, kind, table=BYTES_STEP):
        return (s["segments"] * table[(kind, C)] + s["rays"] * BYTES_RAY(C) +
                s["bvh_nodes"] * BYTES_BOX + s["bvh_faces"] * BYTES_FACE)
    layout = dict(LAYOUT_STEP)
    if acc == "f64":
        layout[("bwd", 1)] = LAYOUT_STEP_ACC64
    dom = "bwd" if bwd_ms >= fwd_ms else "fwd"
    dom_ms = bwd_ms if dom == "bwd" else fwd_ms
    dom_stats = sb if dom == "bwd" else sf
    dom_bytes = alg_bytes(dom_stats, dom)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    bwd_mode = "MODE_BWD64" if acc == "f64" else "MODE_BWD"
    tr = None
    if args.tile == PROFILED_TILE and args.scatter == "atomic" and args.acc == "auto":
        per_seg = profile_per_segment(TRAFFIC_FILE, "dram_bytes_per_segment")
        if per_seg is not None:
            tr = per_seg[dom] * dom_stats["segments"]
    roof = {"bound": "hbm",
            "kernel": f"k_walk32<1,{bwd_mode if dom == 'bwd' else 'MODE_FWD'}> + k_resume32",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": tr, "peak_kind": peak_kind,
            "traffic_note": ("DRAM read+write bytes per call: bytes per segment of an ncu capture on "
                             "the same mesh at 8 angles (profiles/walk32_kuhn96s_traffic.md) x this "
                             "call's segments") if tr is not None
                            else "no capture for this build/configuration",
            "bytes_per_launch": dom_bytes, "ms_per_launch": dom_ms,
            "layout_gbs": alg_bytes(dom_stats, dom, layout) / (dom_ms / 1e3) / 1e9,
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        kind = args.cpu_oracle
        v, cores, dt, ns = cpu_baseline(w, args.cpu_sample or CPU_SAMPLE[kind], kind=kind)
        cpu = {"value": v, "unit": "rays/s", "cores": cores, "kind": "oracle",
               "sample": cpu_sample_text(kind, ns, nrays).replace(" per step", "") + f", {dt:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "nt": mesh.nt, "rays_per_step": nrays,
                   "channels": C, "precision": "filtered", "tile": args.tile,
                   "scatter": args.scatter, "accumulator": acc,
                   "l2": l2_note(mesh.nt, nrays, C),
                   "parallelism": f"replicas{world}"},
        "gsegments_per_s": job_throughput(world, segs, ms_step) / 1e9,
        "segments_per_step": segs,
        "plain_fp64": plain,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "stats": {"fwd": sf, "bwd": sb},
    }
    if args.workload == "cubic64":
        line["adversarial"] = run_adversarial(args, tp, torch, w, mesh, opt, stream)
    return line


def run_adversarial(args, tp, torch, w, mesh, opt, stream):
    """The robustness case's 1M adversarial rays (explicit rays aimed exactly
    at vertices, edge midpoints and face points): forward + backward through
    tetproj_forward_rays / tetproj_backward_rays, filtered and plain FP64."""
    src = torch.tensor(w.extra["adv_src"], device="cuda")
    dst = torch.tensor(w.extra["adv_target"], device="cuda")
    n = src.shape[0]
    out = {}
    for prec, dt in (("filtered", torch.float32), ("plain_fp64", torch.float64)):
        mu = torch.tensor(w.mu, dtype=dt, device="cuda")
        o = tp.make_options(precision=tp.FILTERED if prec == "filtered" else tp.PLAIN_FP64)
        mesh.stats_reset()
        b = tp.forward_rays(mesh, src, dst, mu, options=o)
        tp.backward_rays(mesh, src, dst, b, options=o)
        st = mesh.stats()
        steps = args.steps if prec == "filtered" else 1
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            b = tp.forward_rays(mesh, src, dst, mu, options=o)
            tp.backward_rays(mesh, src, dst, b, options=o)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"value": n / (ms / 1e3), "unit": "rays/s", "ms_per_step": ms, "rays": n,
                     "segments_per_step": st["segments"], "errors": st["error_count"],
                     "sos": st["sos"], "deferred": st["deferred"]}
    return out


def run_recon(args, tp, torch, dist, rank, world, local):
    """The differentiation case: b = A mu_true (plain FP64) + noise, then Adam
    (lr 1e-2) on FP32 mu through TetProject (forward kernel, backward = the
    backprojection kernel).  One step = one Adam iteration."""
    import workloads as W
    w = W.config4()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    b64 = tp.forward(mesh, geo, torch.tensor(w.mu, dtype=torch.float64, device="cuda"))
    sigma = 0.01 * float(b64.max())
    b = (b64 + torch.tensor(w.extra["noise_rng"].normal(0, sigma, size=geo.shape),
                            device="cuda")).float()
    del b64
    mu = torch.zeros(mesh.nt, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([mu], lr=1e-2)
    stream = torch.cuda.current_stream()

    def iteration():
        opt.zero_grad(set_to_none=False)
        r = tp.TetProject.apply(mu, mesh, geo) - b
        loss = 0.5 * (r * r).sum()
        loss.backward()
        opt.step()
        return loss

    for _ in range(args.warmup):
        iteration()
    torch.cuda.synchronize()
    launches0 = tp.launch_count()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            loss = iteration()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = tp.launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    return {
        "metric": METRIC, "value": job_throughput(world, geo.nrays, ms), "unit": "rays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "nt": mesh.nt, "rays_per_step": geo.nrays,
                   "step": "one Adam iteration (forward + backprojection + update)",
                   "parallelism": f"replicas{world}"},
        "ms_per_adam_iteration": ms, "loss": float(loss), "gpu_launches": launches,
        "clocks": clk.summary(),
    }


if __name__ == "__main__":
    main()
