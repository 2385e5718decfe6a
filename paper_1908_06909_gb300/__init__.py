"""GB300-native tetrahedral-mesh CT projectors (thin Python binding).

The compute lives in ``libtetproj.so`` (CUDA, sm_103a) behind the C ABI of
``include/tetproj.h``.  This module only marshals arguments: torch tensors
provide device memory and the current CUDA stream.  There is no CPU
fallback: every call raises if the library or a CUDA device is missing.

Operators (Biguri et al., Sec. II-A):
    forward   b_j = sum_i a_ij mu_i      (Eq. 2)
    backward  x_i = sum_j a_ij y_j       (Eq. 3, the exact adjoint)
with a_ij the length of ray j inside tet i (Eq. 1).  float32 tensors select
the filtered-precision path, float64 tensors the plain FP64 path.

Example::

    import torch
    import paper_1908_06909_gb300 as tp
    from paper_1908_06909_gb300 import solvers
    mesh = tp.Mesh(vertices, tets)          # numpy (nv, 3) float64, (nt, 4) int
    geo = tp.Geometry(dso, dsd, nu, nv, du, dv, angles)   # cone beam, radians
    mu = torch.rand(mesh.nt, device="cuda")               # (nt,) or (nt, 4)
    proj = tp.forward(mesh, geo, mu)                      # [nangles, nv, nu(, 4)]
    back = tp.backward(mesh, geo, proj)                   # [nt(, 4)]
    x = solvers.ossart(mesh, geo, proj, niter=50, block=20)
    # many problems at once: tp.Batch(meshes, geos, channels=4, tiles=...)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (FILTERED, FLAG_ACC32, FLAG_ACC64, FLAG_RSTAR_ENTRY, ORDER_MORTON, ORDER_ROW, PLAIN_FP64,
                   SCATTER_ATOMIC, SCATTER_SORT, SCATTER_WARP, Options, TetprojError, check)

__all__ = ["Mesh", "Geometry", "Batch", "forward", "forward_mt", "forward_rays_mt", "backward", "backward_noalloc", "forward_rays", "backward_rays",
           "trace_rays", "side_signs_host", "side_signs_device", "TetProject", "make_options",
           "FILTERED", "PLAIN_FP64", "ORDER_ROW", "ORDER_MORTON", "SCATTER_ATOMIC",
           "SCATTER_WARP", "SCATTER_SORT", "FLAG_RSTAR_ENTRY", "FLAG_ACC64", "FLAG_ACC32", "entry", "rstar_build_host",
           "TetprojError", "library_path"]


def library_path() -> str:
    return _lib.LIB_PATH


def launch_count() -> int:
    """Kernels the library has launched in this process (host-side count)."""
    return int(_lib.load().tetproj_launch_count())


def version() -> str:
    v = int(_lib.load().tetproj_version())
    return f"{v // 10000}.{v // 100 % 100}.{v % 100}"


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def fma64_peak_tflops(iters: int = 1 << 16, reps: int = 3) -> float:
    """The device's FP64 FMA rate in TFLOP/s, timed with CUDA events around
    tetproj_fma64_probe (best of `reps` launches after one warm-up)."""
    torch = _torch()
    L = _lib.load()
    sink = torch.empty(8 * torch.cuda.get_device_properties(0).multi_processor_count,
                       dtype=torch.float64, device="cuda")
    flops = ctypes.c_double()
    stream = _stream()
    check(L.tetproj_fma64_probe(iters, _ptr(sink), ctypes.byref(flops), stream), "tetproj_fma64_probe")
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        check(L.tetproj_fma64_probe(iters, _ptr(sink), ctypes.byref(flops), stream),
              "tetproj_fma64_probe")
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return flops.value / (best / 1e3) / 1e12


def make_options(precision=FILTERED, channels=1, tile=(16, 8), order=ORDER_MORTON,
                 scatter=SCATTER_ATOMIC, max_steps=0, flags=0) -> Options:
    o = Options()
    _lib.load().tetproj_default_options(ctypes.byref(o))
    o.precision = precision
    o.channels = channels
    o.tile_u, o.tile_v = tile
    o.order = order
    o.scatter = scatter
    o.max_steps = max_steps
    o.flags = flags
    return o


class Mesh:
    """A convex tetrahedral mesh uploaded to the current CUDA device.

    vertices: [nv, 3] float64; tets: [nt, 4] int vertex indices (any
    orientation).  Validation, adjacency, Hilbert renumbering and the boundary
    BVH are built by ``tetproj_mesh_create``."""

    def __init__(self, vertices, tets):
        L = _lib.load()
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        t = np.ascontiguousarray(tets, dtype=np.int32)
        if v.ndim != 2 or v.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 4:
            raise ValueError("vertices must be [nv,3] and tets [nt,4]")
        h = ctypes.c_void_p()
        check(L.tetproj_mesh_create(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0],
                                    ctypes.byref(h)), "tetproj_mesh_create")
        self._h = h
        self.nt = int(t.shape[0])
        self.nv = int(v.shape[0])

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _lib.MeshInfo()
        check(_lib.load().tetproj_mesh_get_info(self._h, ctypes.byref(i)), "tetproj_mesh_get_info")
        d = {k: getattr(i, k) for k, _ in i._fields_ if k != "bbox"}
        d["bbox"] = list(i.bbox)
        return d

    def reserve(self, precision=FILTERED, channels=1):
        check(_lib.load().tetproj_mesh_reserve(self._h, precision, channels), "tetproj_mesh_reserve")

    def stats_reset(self):
        check(_lib.load().tetproj_mesh_stats_reset(self._h, _stream()), "tetproj_mesh_stats_reset")

    def stats(self) -> dict:
        s = _lib.Stats()
        check(_lib.load().tetproj_mesh_stats_read(self._h, _stream(), ctypes.byref(s)),
              "tetproj_mesh_stats_read")
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().tetproj_mesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def topology_host(vertices, tets):
    """(adjacency [nt,4] in input order, nboundary, nflipped), computed on the CPU."""
    L = _lib.load()
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = np.ascontiguousarray(tets, dtype=np.int32)
    adj = np.empty_like(t)
    nb = ctypes.c_int64()
    nf = ctypes.c_int64()
    check(L.tetproj_mesh_topology_host(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0],
                                       adj.ctypes.data, ctypes.byref(nb), ctypes.byref(nf)),
          "tetproj_mesh_topology_host")
    return adj, nb.value, nf.value


class Geometry:
    """Circular cone-beam scan (see include/tetproj.h for the convention)."""

    def __init__(self, dso, dsd, nu, nv, du, dv, angles):
        L = _lib.load()
        a = np.ascontiguousarray(angles, dtype=np.float64)
        h = ctypes.c_void_p()
        check(L.tetproj_geometry_create(float(dso), float(dsd), int(nu), int(nv), float(du),
                                        float(dv), a.ctypes.data, a.size, ctypes.byref(h)),
              "tetproj_geometry_create")
        self._h = h
        self.angles = a.copy()
        self.nu, self.nv, self.nangles = int(nu), int(nv), int(a.size)
        self.dso, self.dsd, self.du, self.dv = float(dso), float(dsd), float(du), float(dv)

    @classmethod
    def from_cone(cls, g):
        """From any object with dso, dsd, nu, nv, du, dv, angles attributes."""
        return cls(g.dso, g.dsd, g.nu, g.nv, g.du, g.dv, g.angles)

    @property
    def handle(self):
        return self._h

    @property
    def nrays(self) -> int:
        return self.nangles * self.nv * self.nu

    @property
    def shape(self):
        return (self.nangles, self.nv, self.nu)

    def rays(self, idx=None, n=None):
        """Device (src, dst) [n, 3] float64 for ray indices (device int64 tensor) or 0..n-1."""
        torch = _torch()
        if idx is not None:
            idx = idx.to(device="cuda", dtype=torch.int64).contiguous()
            n = idx.numel()
        n = self.nrays if n is None else int(n)
        src = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        dst = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        check(_lib.load().tetproj_geometry_rays(self._h, None if idx is None else _ptr(idx), n,
                                                _ptr(src), _ptr(dst), _stream()),
              "tetproj_geometry_rays")
        return src, dst

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().tetproj_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _precision_of(t):
    torch = _torch()
    if t.dtype == torch.float32:
        return FILTERED
    if t.dtype == torch.float64:
        return PLAIN_FP64
    raise TypeError("tensors must be float32 (filtered path) or float64 (plain FP64 path)")


def _check_cuda(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _opts(precision, channels, options):
    o = make_options(precision=precision, channels=channels) if options is None else options
    o.precision = precision
    o.channels = channels
    return o


def forward(mesh: Mesh, geo: Geometry, mu, out=None, options: Options | None = None):
    """proj[a, iv, iu(, c)] = sum_i a_ij mu[i(, c)]  (Eq. 2)."""
    torch = _torch()
    _check_cuda(mu, "mu")
    C = 1 if mu.dim() == 1 else mu.shape[1]
    if mu.shape[0] != mesh.nt:
        raise ValueError("mu must have nt rows")
    prec = _precision_of(mu)
    shape = geo.shape + ((C,) if mu.dim() == 2 else ())
    if out is None:
        out = torch.empty(shape, dtype=mu.dtype, device=mu.device)
    _check_cuda(out, "out")
    o = _opts(prec, C, options)
    check(_lib.load().tetproj_forward(mesh.handle, geo.handle, _ptr(mu), _ptr(out),
                                      ctypes.byref(o), _stream()), "tetproj_forward")
    return out


def backward(mesh: Mesh, geo: Geometry, proj, out=None, options: Options | None = None):
    """mu_out[i(, c)] = sum_j a_ij proj[j(, c)]  (Eq. 3)."""
    torch = _torch()
    _check_cuda(proj, "proj")
    C = 1 if proj.dim() == 3 else proj.shape[3]
    if tuple(proj.shape[:3]) != geo.shape:
        raise ValueError(f"proj must be {geo.shape}(+channels)")
    prec = _precision_of(proj)
    if out is None:
        out = torch.empty((mesh.nt,) + ((C,) if proj.dim() == 4 else ()), dtype=proj.dtype,
                          device=proj.device)
    _check_cuda(out, "out")
    o = _opts(prec, C, options)
    check(_lib.load().tetproj_backward(mesh.handle, geo.handle, _ptr(proj), _ptr(out),
                                       ctypes.byref(o), _stream()), "tetproj_backward")
    return out


def backward_noalloc(mesh: Mesh, geo: Geometry, proj, out=None,
                     options: Options | None = None):
    """tetproj_backward_noalloc: the same A^T y as backward(), with the library's
    fixed device scratch instead of any allocation (see include/tetproj.h for
    its size limit, sharing and first-call rules).  `out` is allocated here by
    torch only when not given."""
    torch = _torch()
    _check_cuda(proj, "proj")
    C = 1 if proj.dim() == 3 else proj.shape[3]
    if tuple(proj.shape[:3]) != geo.shape:
        raise ValueError(f"proj must be {geo.shape}(+channels)")
    prec = _precision_of(proj)
    if out is None:
        out = torch.empty((mesh.nt,) + ((C,) if proj.dim() == 4 else ()), dtype=proj.dtype,
                          device=proj.device)
    _check_cuda(out, "out")
    o = _opts(prec, C, options)
    check(_lib.load().tetproj_backward_noalloc(mesh.handle, geo.handle, _ptr(proj), _ptr(out),
                                               ctypes.byref(o), _stream()),
          "tetproj_backward_noalloc")
    return out


def forward_rays(mesh: Mesh, src, dst, mu, out=None, options: Options | None = None):
    torch = _torch()
    for t, n in ((src, "src"), (dst, "dst"), (mu, "mu")):
        _check_cuda(t, n)
    n = src.shape[0]
    C = 1 if mu.dim() == 1 else mu.shape[1]
    prec = _precision_of(mu)
    if out is None:
        out = torch.empty((n,) + ((C,) if mu.dim() == 2 else ()), dtype=mu.dtype, device=mu.device)
    o = _opts(prec, C, options)
    check(_lib.load().tetproj_forward_rays(mesh.handle, _ptr(src), _ptr(dst), n, _ptr(mu),
                                           _ptr(out), ctypes.byref(o), _stream()),
          "tetproj_forward_rays")
    return out


def backward_rays(mesh: Mesh, src, dst, y, out=None, options: Options | None = None):
    torch = _torch()
    for t, n in ((src, "src"), (dst, "dst"), (y, "y")):
        _check_cuda(t, n)
    C = 1 if y.dim() == 1 else y.shape[1]
    prec = _precision_of(y)
    if out is None:
        out = torch.empty((mesh.nt,) + ((C,) if y.dim() == 2 else ()), dtype=y.dtype,
                          device=y.device)
    o = _opts(prec, C, options)
    check(_lib.load().tetproj_backward_rays(mesh.handle, _ptr(src), _ptr(dst), src.shape[0],
                                            _ptr(y), _ptr(out), ctypes.byref(o), _stream()),
          "tetproj_backward_rays")
    return out


def entry(mesh: Mesh, geo: Geometry, options: Options | None = None):
    """User id of the first tet each cone ray enters (-1: miss), int32
    [na, nv, nu]: the entry search alone (BVH, or the R*-tree with
    FLAG_RSTAR_ENTRY in the options)."""
    torch = _torch()
    out = torch.empty(geo.shape, dtype=torch.int32, device="cuda")
    o = _opts(FILTERED, 1, options)
    check(_lib.load().tetproj_entry(mesh.handle, geo.handle, _ptr(out), ctypes.byref(o),
                                    _stream()), "tetproj_entry")
    return out


def rstar_build_host(vertices, tets) -> dict:
    """Builds the boundary-face R*-tree on the host and checks its invariants."""
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = np.ascontiguousarray(tets, dtype=np.int32)
    info = _lib.RStarInfo()
    check(_lib.load().tetproj_rstar_build_host(v.ctypes.data, v.shape[0], t.ctypes.data,
                                               t.shape[0], ctypes.byref(info)),
          "tetproj_rstar_build_host")
    return {k: getattr(info, k) for k, _ in info._fields_}


def forward_mt(mesh: Mesh, geo: Geometry, mu, options: Options | None = None):
    """The paper's own walk (Alg. 1-2, Moller-Trumbore + growing eps): a
    comparison mode.  float32 mu: single-precision arithmetic, float64: double.
    Returns (proj [na, nv, nu], status int8 [na, nv, nu]: 0 done, 1 halted,
    2 step limit)."""
    torch = _torch()
    _check_cuda(mu, "mu")
    if mu.dim() != 1 or mu.shape[0] != mesh.nt:
        raise ValueError("mu must be [nt]")
    prec = _precision_of(mu)
    out = torch.empty(geo.shape, dtype=mu.dtype, device=mu.device)
    status = torch.empty(geo.shape, dtype=torch.int8, device=mu.device)
    o = _opts(prec, 1, options)
    check(_lib.load().tetproj_forward_mt(mesh.handle, geo.handle, _ptr(mu), _ptr(out),
                                         _ptr(status), ctypes.byref(o), _stream()),
          "tetproj_forward_mt")
    return out, status


def forward_rays_mt(mesh: Mesh, src, dst, mu, options: Options | None = None):
    """forward_mt for explicit rays (device [n, 3] float64 src / dst)."""
    torch = _torch()
    for t, nm in ((src, "src"), (dst, "dst"), (mu, "mu")):
        _check_cuda(t, nm)
    n = src.shape[0]
    prec = _precision_of(mu)
    out = torch.empty((n,), dtype=mu.dtype, device=mu.device)
    status = torch.empty((n,), dtype=torch.int8, device=mu.device)
    o = _opts(prec, 1, options)
    check(_lib.load().tetproj_forward_rays_mt(mesh.handle, _ptr(src), _ptr(dst), n, _ptr(mu),
                                              _ptr(out), _ptr(status), ctypes.byref(o),
                                              _stream()), "tetproj_forward_rays_mt")
    return out, status


def trace_rays(mesh: Mesh, src, dst, max_visits=512, precision=FILTERED,
               options: Options | None = None):
    """Row j of A per ray: (tets [n, max_visits] user ids, lengths, counts)."""
    torch = _torch()
    _check_cuda(src, "src")
    _check_cuda(dst, "dst")
    n = src.shape[0]
    tets = torch.full((n, max_visits), -1, dtype=torch.int32, device="cuda")
    lens = torch.zeros((n, max_visits), dtype=torch.float64, device="cuda")
    cnt = torch.zeros((n,), dtype=torch.int32, device="cuda")
    o = _opts(precision, 1, options)
    check(_lib.load().tetproj_trace_rays(mesh.handle, _ptr(src), _ptr(dst), n, max_visits,
                                         _ptr(tets), _ptr(lens), _ptr(cnt), ctypes.byref(o),
                                         _stream()), "tetproj_trace_rays")
    return tets, lens, cnt


def side_signs_host(S, P, p, q):
    """(sign, stage) of det[P-S, p-S, q-S] via the library's cascade, on the CPU."""
    L = _lib.load()
    arrs = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3) for x in (S, P, p, q)]
    n = arrs[0].shape[0]
    sign = np.zeros(n, np.int8)
    stage = np.zeros(n, np.int8)
    check(L.tetproj_side_host(*[a.ctypes.data for a in arrs], n, sign.ctypes.data,
                              stage.ctypes.data), "tetproj_side_host")
    return sign, stage


def side_signs_device(S, P, p, q):
    """Same cascade evaluated by a CUDA kernel (inputs: device [n,3] float64)."""
    torch = _torch()
    n = S.shape[0]
    sign = torch.zeros(n, dtype=torch.int8, device="cuda")
    stage = torch.zeros(n, dtype=torch.int8, device="cuda")
    check(_lib.load().tetproj_side_device(_ptr(S), _ptr(P), _ptr(p), _ptr(q), n, _ptr(sign),
                                          _ptr(stage), _stream()), "tetproj_side_device")
    return sign, stage


class Batch:
    """Many (mesh, geometry) problems projected by one persistent work-queue
    launch per direction (``tetproj_batch_*``; filtered FP32 path).

    tiles: per problem (tile_u, tile_v, order, scatter), or None for the
    defaults; tiles hold 32..256 rays and may differ between problems.  The
    operand tensors are allocated here (mu/mu_out [nt(,C)], proj/y
    [na, nv, nu(,C)], float32) and bound once, so ``forward()`` and
    ``backward()`` issue stream work only and can be captured in a CUDA graph
    (write new inputs into ``mu[k]`` / ``y[k]`` in place before a replay)."""

    def __init__(self, meshes, geos, channels=1, tiles=None):
        torch = _torch()
        L = _lib.load()
        n = len(meshes)
        if n != len(geos) or n < 1:
            raise ValueError("meshes and geos must be non-empty lists of equal length")
        mh = (ctypes.c_void_p * n)(*[m.handle.value for m in meshes])
        gh = (ctypes.c_void_p * n)(*[g.handle.value for g in geos])
        tl = None
        if tiles is not None:
            t = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(n, 4))
            tl = t
        h = ctypes.c_void_p()
        check(L.tetproj_batch_create(mh, gh, None if tl is None else tl.ctypes.data, n, channels,
                                     ctypes.byref(h)), "tetproj_batch_create")
        self._h = h
        self.meshes, self.geos, self.channels, self.n = list(meshes), list(geos), channels, n
        ext = (channels,) if channels > 1 else ()
        self.mu = [torch.zeros((m.nt,) + ext, dtype=torch.float32, device="cuda") for m in meshes]
        self.mu_out = [torch.zeros((m.nt,) + ext, dtype=torch.float32, device="cuda")
                       for m in meshes]
        self.proj = [torch.zeros(g.shape + ext, dtype=torch.float32, device="cuda") for g in geos]
        self.y = [torch.zeros(g.shape + ext, dtype=torch.float32, device="cuda") for g in geos]
        arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        torch.cuda.synchronize()
        check(L.tetproj_batch_bind(self._h, arr(self.mu), arr(self.proj), arr(self.y),
                                   arr(self.mu_out)), "tetproj_batch_bind")

    @property
    def nrays(self) -> int:
        return sum(g.nrays for g in self.geos)

    def forward(self):
        """proj[k] = A_k mu[k] for every problem (async on the current stream)."""
        check(_lib.load().tetproj_batch_forward(self._h, _stream()), "tetproj_batch_forward")
        return self.proj

    def backward(self):
        """mu_out[k] = A_k^T y[k] for every problem (async on the current stream)."""
        check(_lib.load().tetproj_batch_backward(self._h, _stream()), "tetproj_batch_backward")
        return self.mu_out

    def set_wait(self, max_polls: int = 0, never_satisfied: bool = False):
        """tetproj_batch_set_wait: the poll bound of the persistent kernel's
        inter-warp waits (0: the default); never_satisfied makes every wait run
        out (a test of the timeout path)."""
        check(_lib.load().tetproj_batch_set_wait(self._h, int(max_polls), int(bool(never_satisfied))),
              "tetproj_batch_set_wait")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().tetproj_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_cls():
    torch = _torch()

    class _TetProject(torch.autograd.Function):
        """proj = A mu with backward g -> A^T g (the hand-written backprojection)."""

        @staticmethod
        def forward(ctx, mu, mesh, geo, options):
            ctx.mesh, ctx.geo, ctx.options = mesh, geo, options
            return forward(mesh, geo, mu.contiguous(), options=options)

        @staticmethod
        def backward(ctx, g):
            gmu = backward(ctx.mesh, ctx.geo, g.contiguous(), options=ctx.options)
            return gmu, None, None, None

    return _TetProject


_TP = None


class TetProject:
    """``TetProject.apply(mu, mesh, geo, options=None)``: differentiable A mu."""

    @staticmethod
    def apply(mu, mesh, geo, options=None):
        global _TP
        if _TP is None:
            _TP = _autograd_cls()
        return _TP.apply(mu, mesh, geo, options)
