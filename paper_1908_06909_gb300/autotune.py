"""Launch-shape autotuner for the projectors.

The paper picked its GPU block sizes by trying several and keeping the
fastest (Sec. II-F).  This module does the same per *size class* of problem
and caches the result on disk:

* space: ray tile (tile_u x tile_v threads per CTA), tile ordering (row-major
  or Morton inside the tile) and backprojection scatter (plain atomics,
  warp-aggregated atomics, or the deterministic segment sort-and-reduce; the
  batched launch adds atomically, so batches choose between the first two);
* size class: (ceil log2 of the tet count, ceil log2 of the detector pixel
  count, channels, threads per CTA or "any");
* measurement: forward + backward on a reduced scan of the problem itself (a
  few of its angles, at most ~2M rays), timed with CUDA events on the current
  stream after one warm-up, median of `reps`, in ms per million rays.  Tile
  and ordering are chosen on forward + backward time with atomic scatter,
  then the scatter on backward time with that tile.

``tune_batch`` returns per-problem (tile_u, tile_v, order, scatter) rows for
``Batch(..., tiles=...)``: the batched kernel hands out 32-ray warp slices of
tiles, so every problem may use its own tile of at least 32 rays.

The cache is JSON keyed by device name, library version and size class; its
path is ``$TETPROJ_TUNE_CACHE`` or ``~/.cache/tetproj/autotune.json``.  The
search itself is plain host logic over a measuring callback (tested on the CPU
with a synthetic timer).
"""
from __future__ import annotations

import json
import math
import os
import statistics
from dataclasses import dataclass

ORDER_ROW = 0
ORDER_MORTON = 1
SCATTER_ATOMIC = 0
SCATTER_WARP = 1

# tiles per thread count (the row-major-friendly wide tile first); every tile
# holds whole warps (a 4 x 4 tile would leave half of each warp without a ray)
TILES = {
    32: [(8, 4), (4, 8)],
    64: [(8, 8), (16, 4), (4, 16)],
    128: [(16, 8), (8, 16), (32, 4)],
    256: [(16, 16), (32, 8)],
}
SCATTER_SORT = 2
ORDERS = (ORDER_MORTON, ORDER_ROW)
SCATTERS = (SCATTER_ATOMIC, SCATTER_WARP, SCATTER_SORT)
BATCH_SCATTERS = (SCATTER_ATOMIC, SCATTER_WARP)  # the batched launch adds atomically
MAX_TUNE_RAYS = 2_000_000
BATCH_MIN_THREADS = 32  # the batched kernel walks 32-ray slices of a tile


@dataclass(frozen=True)
class Choice:
    tile_u: int
    tile_v: int
    order: int
    scatter: int

    def row(self):
        return (self.tile_u, self.tile_v, self.order, self.scatter)


def size_class(nt: int, npix: int, channels: int, threads: int | None,
               min_threads: int = 32) -> str:
    """Cache key of a problem: log2 buckets of tets and detector pixels."""
    a = max(0, math.ceil(math.log2(max(nt, 1))))
    b = max(0, math.ceil(math.log2(max(npix, 1))))
    n = threads if threads else ("any" if min_threads <= 32 else f"ge{min_threads}")
    return f"t{a}_p{b}_c{channels}_n{n}"


def candidates(threads: int | None = None, min_threads: int = 32):
    """(tile_u, tile_v, order) candidates: tiles of `threads` threads, or of
    every count >= min_threads if threads is None."""
    counts = [n for n in sorted(TILES) if n >= min_threads] if threads is None else [threads]
    out = []
    for n in counts:
        if n not in TILES:
            raise ValueError(f"no tiles with {n} threads")
        for t in TILES[n]:
            for o in ORDERS:
                out.append((t[0], t[1], o))
    return out


def search(measure, threads: int | None = None, min_threads: int = 32, scatters=SCATTERS):
    """Pick (Choice, best_ms) with measure(Choice, what) -> ms, what in
    {"fwd+bwd", "bwd"}: tile/order on fwd+bwd with atomic scatter, then the
    scatter among `scatters` on bwd with the chosen tile."""
    best, best_ms = None, math.inf
    for tu, tv, o in candidates(threads, min_threads):
        c = Choice(tu, tv, o, SCATTER_ATOMIC)
        ms = measure(c, "fwd+bwd")
        if ms < best_ms:
            best, best_ms = c, ms
    bwd = {s: measure(Choice(best.tile_u, best.tile_v, best.order, s), "bwd") for s in scatters}
    s = min(bwd, key=lambda k: (bwd[k], k))
    if s != best.scatter:
        best_ms += bwd[s] - bwd[best.scatter]
        best = Choice(best.tile_u, best.tile_v, best.order, s)
    return best, best_ms


class Cache:
    """JSON file {device|version: {size_class: {"choice": [...], "ms": t}}},
    t in ms per million rays."""

    def __init__(self, path: str | None = None, device: str = "", version: str = ""):
        self.path = path or os.environ.get("TETPROJ_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "tetproj", "autotune.json")
        self.scope = f"{device}|{version}"
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key: str):
        e = self.data.get(self.scope, {}).get(key)
        if not e:
            return None
        return Choice(*e["choice"]), float(e["ms"])

    def put(self, key: str, choice: Choice, ms: float):
        self.data.setdefault(self.scope, {})[key] = {"choice": list(choice.row()), "ms": ms}

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tune_problem(key: str, make_measure, threads: int | None, cache: Cache | None,
                 min_threads: int = 32, scatters=SCATTERS):
    """(Choice, ms) for a size class: from the cache, else by search() over the
    callback make_measure() returns (built only on a cache miss)."""
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            return hit
    choice, ms = search(make_measure(), threads, min_threads, scatters)
    if cache is not None:
        cache.put(key, choice, ms)
    return choice, ms


# ----------------------------------------------------------- GPU measuring


def _reduced_geometry(tp, geo):
    import numpy as np
    npix = geo.nu * geo.nv
    na = max(1, min(8, geo.nangles, MAX_TUNE_RAYS // max(npix, 1)))
    ang = np.asarray(_angles_of(geo), dtype=np.float64)
    sel = ang[np.linspace(0, ang.size - 1, na).round().astype(int)]
    return tp.Geometry(geo.dso, geo.dsd, geo.nu, geo.nv, geo.du, geo.dv, sel)


def _angles_of(geo):
    a = getattr(geo, "angles", None)
    if a is None:
        raise ValueError("geometry has no angle list (construct it with Geometry(...))")
    return a


def gpu_measure(tp, mesh, geo, channels: int, reps: int = 3):
    """A measure(Choice, what) callback timing tp.forward/backward (float32,
    filtered path) on a reduced scan of (mesh, geo); returns ms per Mray."""
    import torch
    g = _reduced_geometry(tp, geo)
    ext = (channels,) if channels > 1 else ()
    gen = torch.Generator(device="cuda").manual_seed(12345)
    mu = torch.rand((mesh.nt,) + ext, device="cuda", generator=gen)
    y = torch.rand(g.shape + ext, device="cuda", generator=gen)
    proj = torch.empty_like(y)
    back = torch.empty_like(mu)

    def measure(c: Choice, what: str) -> float:
        o = tp.make_options(precision=tp.FILTERED, channels=channels,
                            tile=(c.tile_u, c.tile_v), order=c.order, scatter=c.scatter)

        def run():
            if what == "fwd+bwd":
                tp.forward(mesh, g, mu, out=proj, options=o)
            tp.backward(mesh, g, y, out=back, options=o)

        run()
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return statistics.median(times) / (g.nrays / 1e6)

    return measure


def _cache_for(tp, cache):
    if cache is False:
        return None
    if isinstance(cache, Cache):
        return cache
    import torch
    return Cache(cache, device=torch.cuda.get_device_name(), version=tp.version())


def tune(tp, mesh, geo, channels: int = 1, threads: int | None = None, cache=None,
         reps: int = 3) -> Choice:
    """Best Choice for one (mesh, geometry); cache=False disables the cache."""
    c = _cache_for(tp, cache)
    key = size_class(mesh.nt, geo.nu * geo.nv, channels, threads)
    choice, _ = tune_problem(key, lambda: gpu_measure(tp, mesh, geo, channels, reps), threads, c)
    if c is not None:
        c.save()
    return choice


def tune_batch(tp, meshes, geos, channels: int = 1, cache=None, reps: int = 3):
    """[Choice per problem] for a Batch over (meshes[k], geos[k]): each
    problem's best tile of at least 32 rays (problems of one size class share
    one measurement through the cache)."""
    c = _cache_for(tp, cache) if cache is not False else None
    memo = {}
    out = []
    for m, g in zip(meshes, geos):
        key = size_class(m.nt, g.nu * g.nv, channels, None,
                         min_threads=BATCH_MIN_THREADS) + "_batch"
        if key not in memo:
            memo[key] = tune_problem(key, lambda m=m, g=g: gpu_measure(tp, m, g, channels, reps),
                                     None, c, min_threads=BATCH_MIN_THREADS,
                                     scatters=BATCH_SCATTERS)[0]
        out.append(memo[key])
    if c is not None:
        c.save()
    return out
