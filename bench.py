#!/usr/bin/env python
"""Benchmark: forward + back projection on the jittered Kuhn 96^3 workload.

One step = tetproj_forward (b = A mu) followed by tetproj_backward of that
projection (x = A^T b): 512 x 512 x 360 = 94,371,840 cone-beam rays through
5,308,416 tets, each way.  `value` is rays/s of such fwd+back pairs on the
device (inputs resident in HBM); `e2e` is the same through the C ABI with host
buffers (pinned H2D of mu, D2H of the projection and the backprojection every
step).  The filtered FP32 path is the product; the plain FP64 path is timed
beside it for the ratio.  Under torchrun every rank runs an independent
replica (the operator shards over rays with no exchange in the forward; this
build has no cross-GPU step), so value = all ranks' rays / max time.

--impl reference times the CPU oracle (brute-force FP64 clipping) on a bounded
sample of the same rays, on the host cores.
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


def cpu_baseline(w, nsample, threads=None):
    """The oracle as it stands, on `nsample` rays spread over the workload:
    forward (b_j for the sampled rays) and backward (A^T y restricted to
    those rays); returns fwd+back ray pairs per second."""
    import oracle
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(w.geom.nrays, nsample, replace=False))
    S, P = oracle.cone_rays(w.geom, idx)
    y = rng.uniform(size=nsample)
    threads = threads or oracle.default_threads()
    t0 = time.perf_counter()
    oracle.forward_rays(w.verts, w.tets, w.mu, S, P, threads=threads)
    oracle.backward_rays(w.verts, w.tets, y, S, P, threads=threads)
    dt = time.perf_counter() - t0
    return nsample / dt, threads, dt, idx.size


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = build_workload(args)
    n = args.cpu_sample
    for _ in range(args.warmup):
        cpu_baseline(w, max(8, n // 16))
    times = []
    for _ in range(args.steps):
        v, cores, dt, ns = cpu_baseline(w, n)
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
                         "sample": f"{n} of {w.geom.nrays} rays per step (fwd + back), brute-force FP64 clipping over all tets"},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kuhn96")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--scatter", default="atomic", choices=["atomic", "warp"])
    ap.add_argument("--tile", default="8x8")
    args = ap.parse_args()

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

    w = build_workload(args)
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    tu, tv = (int(x) for x in args.tile.split("x"))
    opt = tp.make_options(tile=(tu, tv), scatter=tp.SCATTER_WARP if args.scatter == "warp"
                          else tp.SCATTER_ATOMIC)
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
    if dist:
        dist.barrier()
    total_ms = start.elapsed_time(end)
    fwd_ms = float(np.mean([a.elapsed_time(b) for a, b, _ in evs]))
    bwd_ms = float(np.mean([b.elapsed_time(c) for _, b, c in evs]))
    t = torch.tensor([total_ms], device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item()) / args.steps
    nrays = geo.nrays
    value = world * nrays / (ms_step / 1e3)
    segs = sf["segments"] + sb["segments"]

    # plain FP64 path (the ratio's denominator), same step
    plain = None
    if args.plain_steps > 0:
        mu64 = mu.double()
        proj64 = torch.empty(geo.shape, dtype=torch.float64, device="cuda")
        back64 = torch.empty(mesh.nt, dtype=torch.float64, device="cuda")
        o64 = tp.make_options(precision=tp.PLAIN_FP64, tile=(tu, tv), scatter=opt.scatter)
        tp.forward(mesh, geo, mu64, out=proj64, options=o64)
        tp.backward(mesh, geo, proj64, out=back64, options=o64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.plain_steps):
            tp.forward(mesh, geo, mu64, out=proj64, options=o64)
            tp.backward(mesh, geo, proj64, out=back64, options=o64)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b) / args.plain_steps
        rel = float(((proj.double() - proj64).abs().sum() / proj64.abs().sum()).item())
        plain = {"value": nrays / (pms / 1e3), "unit": "rays/s", "ms_per_step": pms,
                 "speedup_filtered_vs_plain": (nrays / (ms_step / 1e3)) / (nrays / (pms / 1e3)),
                 "filtered_vs_plain_rel_l1_diff": rel}
        del proj64, back64, mu64

    # end to end through the public API with host buffers
    mu_h = torch.empty(mesh.nt, dtype=torch.float32, pin_memory=True)
    mu_h.copy_(mu.cpu())
    proj_h = torch.empty(geo.shape, dtype=torch.float32, pin_memory=True)
    back_h = torch.empty(mesh.nt, dtype=torch.float32, pin_memory=True)
    mu_d = torch.empty_like(mu)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        mu_d.copy_(mu_h, non_blocking=True)
        tp.forward(mesh, geo, mu_d, out=proj, options=opt)
        tp.backward(mesh, geo, proj, out=back, options=opt)
        proj_h.copy_(proj, non_blocking=True)
        back_h.copy_(back, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / args.steps
    te = torch.tensor([e2e_ms], device="cuda")
    if dist:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": world * nrays / (float(te.item()) / 1e3), "unit": "rays/s",
           "h2d_bytes_per_step": mu_h.numel() * 4,
           "d2h_bytes_per_step": proj_h.numel() * 4 + back_h.numel() * 4}

    # roofline of the dominant walk (events around each call; the O(nt)
    # permutation kernels inside the call are < 0.1% of it)
    hbm, peak_kind = peaks()
    def alg_bytes(s, kind, table=BYTES_STEP):
        return (s["segments"] * table[(kind, C)] + s["rays"] * BYTES_RAY(C) +
                s["bvh_nodes"] * BYTES_BOX + s["bvh_faces"] * BYTES_FACE)
    dom = "bwd" if bwd_ms >= fwd_ms else "fwd"
    dom_ms = bwd_ms if dom == "bwd" else fwd_ms
    dom_bytes = alg_bytes(sb if dom == "bwd" else sf, dom)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": f"k_walk32<1,{'MODE_BWD' if dom == 'bwd' else 'MODE_FWD'}>",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "peak_kind": peak_kind,
            "bytes_per_launch": dom_bytes, "ms_per_launch": dom_ms,
            "layout_gbs": alg_bytes(sb if dom == "bwd" else sf, dom, LAYOUT_STEP) / (dom_ms / 1e3) / 1e9,
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        v, cores, dt, ns = cpu_baseline(w, args.cpu_sample)
        cpu = {"value": v, "unit": "rays/s", "cores": cores, "kind": "oracle",
               "sample": f"{ns} of {nrays} rays (fwd + back), brute-force FP64 clipping, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "nt": mesh.nt, "rays_per_step": nrays,
                       "channels": C, "precision": "filtered", "tile": args.tile,
                       "scatter": args.scatter,
                       "l2": "inputs larger than L2 (tet records 340 MB, projections 377 MB)",
                       "parallelism": f"replicas{world}"},
            "gsegments_per_s": world * segs / (ms_step / 1e3) / 1e9,
            "segments_per_step": segs,
            "plain_fp64": plain,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 4 * args.steps,
            "clocks": clk.summary(),
            "stats": {"fwd": sf, "bwd": sb},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
