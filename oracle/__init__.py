"""CPU oracle for the tetrahedral-mesh projectors -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` and ``--impl reference`` legs) may import this package.  The
product library never loads it, and it shares no code with the CUDA path.

``oracle.c`` evaluates the paper's plain definition (Eq. 1-3): every chord
a_ij = |half-line j  intersected with closed tet i| is computed by brute-force
clipping of every ray against every tet, in FP64.  Its walker (``Walker``)
gives the same a_ij, each from the same clipping code, for the tets a ray
passes through, found over adjacency the oracle builds itself (rays with
near-ties get the brute-force row), so that large samples are affordable.
``exact.py`` holds exact rational predicates (orientation, the symbolic
tie-break) used to pin the predicate cascade of the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_MT = os.path.join(_HERE, "mt.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_ip = ctypes.POINTER(ctypes.c_int32)
_c_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, FP64, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_MT))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", "-o", tmp, _SRC, _SRC_MT, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_version.restype = ctypes.c_int64
        L.oracle_cone_rays.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_double, ctypes.c_double, _c_dp,
                                       ctypes.c_int64, _c_lp, ctypes.c_int64, _c_dp, _c_dp]
        L.oracle_mt_forward_rays.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64, _c_dp,
                                             _c_dp, _c_dp, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_int64, _c_dp,
                                             ctypes.POINTER(ctypes.c_int8)]
        L.oracle_tet_chord.argtypes = [_c_dp, _c_dp, _c_dp, _c_dp, _c_dp]
        L.oracle_tet_chord.restype = ctypes.c_double
        L.oracle_forward_rays.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64, _c_dp,
                                          ctypes.c_int, _c_dp, _c_dp, _c_dp, ctypes.c_int64,
                                          _c_dp, ctypes.c_int]
        L.oracle_forward_rays_range.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64,
                                                _c_dp, ctypes.c_int, _c_dp, _c_dp, _c_dp, _c_dp,
                                                _c_dp, ctypes.c_int64, _c_dp, ctypes.c_int]
        L.oracle_forward_cone.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64, _c_dp,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_double, _c_dp, ctypes.c_int64, _c_lp,
                                          ctypes.c_int64, _c_dp, ctypes.c_int]
        L.oracle_backward_rays.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64, _c_dp,
                                           ctypes.c_int, _c_dp, _c_dp, _c_dp, ctypes.c_int64,
                                           _c_dp, ctypes.c_int]
        L.oracle_backward_cone.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64, _c_dp,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_double, _c_dp, ctypes.c_int64, _c_dp,
                                           ctypes.c_int]
        L.oracle_backward_cone_subset.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64,
                                                  _c_dp, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_double, ctypes.c_double, _c_dp,
                                                  ctypes.c_int64, _c_lp, ctypes.c_int64, _c_dp,
                                                  ctypes.c_int]
        L.oracle_trace_rays.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64, _c_dp,
                                        _c_dp, ctypes.c_int64, ctypes.c_int64, _c_ip, _c_dp,
                                        _c_dp, _c_lp, _c_dp, _c_ip, ctypes.c_int]
        L.oracle_walker_create.argtypes = [_c_dp, ctypes.c_int64, _c_ip, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int)]
        L.oracle_walker_create.restype = ctypes.c_void_p
        L.oracle_walker_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_walker_destroy.restype = None
        L.oracle_walk.argtypes = [ctypes.c_void_p, _c_dp, _c_dp, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_double, ctypes.c_double, _c_dp, ctypes.c_int64,
                                  _c_lp, _c_dp, _c_dp, ctypes.c_int64, _c_dp, _c_dp, _c_lp,
                                  ctypes.c_double, _c_dp, _c_dp,
                                  ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        L.oracle_walk.restype = ctypes.c_int
        L.oracle_walk_trace.argtypes = [ctypes.c_void_p, _c_dp, _c_dp, ctypes.c_int64,
                                        ctypes.c_int64, _c_ip, _c_dp, _c_dp, _c_lp,
                                        ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        L.oracle_walk_trace.restype = ctypes.c_int
        for f in ("oracle_forward_rays", "oracle_forward_rays_range", "oracle_forward_cone", "oracle_backward_rays",
                  "oracle_backward_cone", "oracle_backward_cone_subset", "oracle_trace_rays"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_c_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_c_ip)


def _l(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_c_lp)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def cone_rays(geom, idx=None):
    """(S, P) endpoints [n,3] for cone-beam ray indices j = (a*nv + iv)*nu + iu."""
    ang, angp = _d(geom.angles)
    n = geom.nrays if idx is None else len(idx)
    S = np.empty((n, 3))
    P = np.empty((n, 3))
    if idx is None:
        ip = None
    else:
        idx, ip = _l(idx)
    lib().oracle_cone_rays(geom.dso, geom.dsd, geom.nu, geom.nv, geom.du, geom.dv, angp,
                           geom.nangles, ip, n, S.ctypes.data_as(_c_dp), P.ctypes.data_as(_c_dp))
    return S, P


def tet_chord(tet_verts, S, P):
    """a for one tet [4,3] and one ray; returns (length, t_lo, t_hi)."""
    v, vp = _d(np.asarray(tet_verts).reshape(12))
    s, sp = _d(S)
    p, pp = _d(P)
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    a = lib().oracle_tet_chord(vp, sp, pp, ctypes.byref(lo), ctypes.byref(hi))
    return a, lo.value, hi.value


def _mesh(verts, tets):
    v, vp = _d(verts)
    t, tp = _i(tets)
    return v, vp, t, tp


def _channels(x, n):
    x = np.asarray(x, dtype=np.float64)
    C = 1 if x.ndim == 1 else x.shape[1]
    return np.ascontiguousarray(x.reshape(n, C)), C


def forward_rays(verts, tets, mu, S, P, side=None, threads=None):
    """b_j = sum_i a_ij mu_i for explicit rays (Eq. 2).  ``side``: per-ray
    directions [n,3] choosing one-sided limits for rays in face planes."""
    v, vp, t, tp = _mesh(verts, tets)
    mu2, C = _channels(mu, t.shape[0])
    m, mp = _d(mu2)
    s, sp = _d(S)
    p, pp = _d(P)
    n = s.shape[0]
    w, wp = (None, None) if side is None else _d(side)
    out = np.empty((n, C))
    _check(lib().oracle_forward_rays(vp, v.shape[0], tp, t.shape[0], mp, C, sp, pp, wp, n,
                                     out.ctypes.data_as(_c_dp), threads or default_threads()),
           "oracle_forward_rays")
    return out[:, 0] if np.asarray(mu).ndim == 1 else out


def forward_rays_range(verts, tets, mu, S, P, t0, t1, side=None, threads=None):
    """b_j restricted to parameters t in [t0_j, t1_j] (t1 may be inf)."""
    v, vp, t, tp = _mesh(verts, tets)
    mu2, C = _channels(mu, t.shape[0])
    m, mp = _d(mu2)
    s, sp = _d(S)
    p, pp = _d(P)
    n = s.shape[0]
    a0, a0p = _d(np.broadcast_to(np.asarray(t0, float), (n,)))
    a1, a1p = _d(np.broadcast_to(np.asarray(t1, float), (n,)))
    w, wp = (None, None) if side is None else _d(side)
    out = np.empty((n, C))
    _check(lib().oracle_forward_rays_range(vp, v.shape[0], tp, t.shape[0], mp, C, sp, pp, wp, a0p,
                                           a1p, n, out.ctypes.data_as(_c_dp),
                                           threads or default_threads()),
           "oracle_forward_rays_range")
    return out[:, 0] if np.asarray(mu).ndim == 1 else out


def sos_side_direction():
    """A concrete direction ordered like the symbolic perturbation of the ray
    source (e, e^2, e^4): its sign against a plane normal n is that of the first
    non-zero component of n whenever the components of n are not below 1e-6 of
    the leading one.  ``forward_rays_exact_planar`` checks that condition, in
    exact arithmetic, for every plane it uses the direction on."""
    return np.array([1.0, 1e-6, 1e-12])


class PlanarSideError(ValueError):
    """The concrete side direction does not reproduce the symbolic side."""


def check_side_direction(normals, w=None):
    """Raise PlanarSideError unless, for every exact integer plane normal n,
    n . w has the sign of the first non-zero component of n by more than the
    FP64 error of the clipper's own n . w.  ``normals`` is a list of integer
    triples (their cross products taken as exact) or the dict {normal: E} of
    exact.face_planes_containing: the clipper's normal is a cross product of
    FP64 edge vectors, off by at most ~4 u E_k in component k (nothing where
    both of its products are exactly zero), and its dot product with w adds
    ~3 u sum |n_k w_k|."""
    from fractions import Fraction as Fr
    from oracle import exact
    u = 2.0 ** -53
    w = sos_side_direction() if w is None else np.asarray(w, float)
    wf = [Fr(float(x)) for x in w]
    bound = normals if isinstance(normals, dict) else {tuple(n): (0.0, 0.0, 0.0) for n in normals}
    for n, E in bound.items():
        want = exact.sos_side_sign(n)
        dot = sum(Fr(int(a)) * b for a, b in zip(n, wf))
        err = sum(8.0 * u * E[k] * abs(float(w[k])) + 4.0 * u * abs(int(n[k]) * float(w[k]))
                  for k in range(3))
        if want == 0 or exact.sign(dot) != want or abs(float(dot)) <= err:
            raise PlanarSideError(f"side direction {w} does not reproduce the symbolic "
                                  f"side of the plane with normal {n}")


def forward_rays_exact_planar(verts, tets, mu, S, P, threads=None):
    """Integral of rays lying EXACTLY in a face plane, as the limit of the
    symbolically perturbed line S + (e, e^2, e^4), P + (e^8, ...): on [0, 1) the
    line sits on the side of the source perturbation, beyond t = 1 (the point P)
    on the opposite side.  The side is realised by a concrete direction
    (``sos_side_direction``); every plane containing each ray is found exactly
    and the direction is checked against the symbolic sign first.  Raises
    PlanarSideError for a ray in no face plane, or where the direction would
    pick the wrong side."""
    from oracle import exact
    S = np.atleast_2d(np.asarray(S, float))
    P = np.atleast_2d(np.asarray(P, float))
    n = S.shape[0]
    for k in range(n):
        normals = exact.face_planes_containing(verts, tets, S[k], P[k], return_kappa=True)
        if not normals:
            raise PlanarSideError(f"ray {k} lies in no face plane")
        check_side_direction(normals)
    w = np.broadcast_to(sos_side_direction(), (n, 3)).copy()
    a = forward_rays_range(verts, tets, mu, S, P, 0.0, 1.0, side=w, threads=threads)
    b = forward_rays_range(verts, tets, mu, S, P, 1.0, np.inf, side=-w, threads=threads)
    return a + b


def forward_cone(verts, tets, mu, geom, ray_idx=None, threads=None):
    """b = A mu for cone-beam rays (all, or the selected ray indices)."""
    v, vp, t, tp = _mesh(verts, tets)
    mu2, C = _channels(mu, t.shape[0])
    m, mp = _d(mu2)
    ang, angp = _d(geom.angles)
    if ray_idx is None:
        ip, n = None, geom.nrays
    else:
        ray_idx, ip = _l(ray_idx)
        n = ray_idx.size
    out = np.empty((n, C))
    _check(lib().oracle_forward_cone(vp, v.shape[0], tp, t.shape[0], mp, C, geom.dso, geom.dsd,
                                     geom.nu, geom.nv, geom.du, geom.dv, angp, geom.nangles, ip, n,
                                     out.ctypes.data_as(_c_dp), threads or default_threads()),
           "oracle_forward_cone")
    return out[:, 0] if np.asarray(mu).ndim == 1 else out


def backward_rays(verts, tets, y, S, P, side=None, threads=None):
    """x_i = sum_j a_ij y_j for explicit rays (Eq. 3)."""
    v, vp, t, tp = _mesh(verts, tets)
    s, sp = _d(S)
    n = s.shape[0]
    y2, C = _channels(y, n)
    yy, yp = _d(y2)
    p, pp = _d(P)
    w, wp = (None, None) if side is None else _d(side)
    out = np.empty((t.shape[0], C))
    _check(lib().oracle_backward_rays(vp, v.shape[0], tp, t.shape[0], yp, C, sp, pp, wp, n,
                                      out.ctypes.data_as(_c_dp), threads or default_threads()),
           "oracle_backward_rays")
    return out[:, 0] if np.asarray(y).ndim == 1 else out


def backward_cone(verts, tets, y, geom, threads=None):
    """x = A^T y over all cone-beam rays; y laid out [angle][iv][iu](,C)."""
    v, vp, t, tp = _mesh(verts, tets)
    y = np.asarray(y, dtype=np.float64)
    C = y.size // geom.nrays
    y2 = y.reshape(geom.nrays, C)
    yy, yp = _d(y2)
    ang, angp = _d(geom.angles)
    out = np.empty((t.shape[0], C))
    _check(lib().oracle_backward_cone(vp, v.shape[0], tp, t.shape[0], yp, C, geom.dso, geom.dsd,
                                      geom.nu, geom.nv, geom.du, geom.dv, angp, geom.nangles,
                                      out.ctypes.data_as(_c_dp), threads or default_threads()),
           "oracle_backward_cone")
    return out[:, 0] if C == 1 else out


def backward_cone_subset(verts, tets, y, geom, tet_idx, threads=None):
    """x_i for the selected tets only, summed over all cone-beam rays."""
    v, vp, t, tp = _mesh(verts, tets)
    y = np.asarray(y, dtype=np.float64)
    C = 1 if y.size == geom.nrays else y.size // geom.nrays
    yy, yp = _d(y.reshape(geom.nrays, C))
    ang, angp = _d(geom.angles)
    tet_idx, ip = _l(tet_idx)
    out = np.empty((tet_idx.size, C))
    _check(lib().oracle_backward_cone_subset(vp, v.shape[0], tp, t.shape[0], yp, C, geom.dso,
                                             geom.dsd, geom.nu, geom.nv, geom.du, geom.dv, angp,
                                             geom.nangles, ip, tet_idx.size,
                                             out.ctypes.data_as(_c_dp),
                                             threads or default_threads()),
           "oracle_backward_cone_subset")
    return out[:, 0] if C == 1 else out


class Walker:
    """Rows of A found by walking face adjacency (the oracle walker of
    ``oracle.c``): the same a_ij as the brute-force clipper, each computed by
    the same clipping code, but only for the tets a ray passes through.  Rays
    with a near-tie anywhere on their walk (two candidate entries or exits
    within 1e-9 in t, a visit shorter than that, a face plane containing the
    ray) get the brute-force row instead.  The adjacency is the oracle's own,
    built from the vertex ids.  Meant for convex meshes with sources outside;
    any other ray still gets a brute-force row."""

    def __init__(self, verts, tets):
        self._v, vp = _d(verts)
        self._t, tp = _i(tets)
        st = ctypes.c_int(0)
        h = lib().oracle_walker_create(vp, self._v.shape[0], tp, self._t.shape[0], ctypes.byref(st))
        if not h:
            raise RuntimeError(f"oracle_walker_create failed with code {st.value}")
        self._h = ctypes.c_void_p(h)
        self.nt = self._t.shape[0]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_walker_destroy(h)
            self._h = None

    def _run(self, mu, y, geom, ray_idx, S, P, threads, cap=64.0, cond=True):
        if S is not None:
            s, sp = _d(S)
            p, pp = _d(P)
            n = s.shape[0]
            ip, angp, g = None, None, (0.0, 0.0, 0, 0, 0.0, 0.0)
            na = 0
        else:
            sp = pp = None
            ray_idx, ip = _l(np.arange(geom.nrays) if ray_idx is None else ray_idx)
            n = ray_idx.size
            ang, angp = _d(geom.angles)
            g = (geom.dso, geom.dsd, geom.nu, geom.nv, geom.du, geom.dv)
            na = geom.nangles
        mp = yp = None
        C = 1
        if mu is not None:
            mu2, C = _channels(mu, self.nt)
            m, mp = _d(mu2)
        if y is not None:
            y2, C = _channels(y, n)
            yy, yp = _d(y2)
        fwd = np.empty((n, C)) if mu is not None else None
        bwd = np.empty((self.nt, C)) if y is not None else None
        cnt = np.empty(self.nt, dtype=np.int64) if y is not None else None
        kf = np.empty((n, C, 2)) if (cond and mu is not None) else None
        kb = np.empty((self.nt, C, 2)) if (cond and y is not None) else None
        status = np.empty(n, dtype=np.int8)
        ptr = lambda a, t=_c_dp: None if a is None else a.ctypes.data_as(t)
        _check(lib().oracle_walk(self._h, mp, yp, C, *g, angp, na, ip, sp, pp, n, ptr(fwd),
                                 ptr(bwd), ptr(cnt, _c_lp), float(cap), ptr(kf), ptr(kb),
                                 status.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                 threads or default_threads()), "oracle_walk")
        self.last_count, self.last_kf, self.last_kb = cnt, kf, kb
        return fwd, bwd, status

    def forward_cone(self, mu, geom, ray_idx=None, threads=None):
        """(b [n](,C), status [n]) for the selected cone rays (Eq. 2);
        status 0 walked, 1 brute force, 2 brute force, ray in a face plane."""
        fwd, _, st = self._run(mu, None, geom, ray_idx, None, None, threads, cond=False)
        return (fwd[:, 0] if np.asarray(mu).ndim == 1 else fwd), st

    def backward_cone(self, y, geom, ray_idx, threads=None):
        """(x [nt](,C), status): x_i = sum_k a_i,ray_idx[k] y[k] (Eq. 3 over
        the selected cone rays only).  ``last_count`` then holds, per tet, how
        many of these rays cross it."""
        _, bwd, st = self._run(None, y, geom, ray_idx, None, None, threads, cond=False)
        return (bwd[:, 0] if np.asarray(y).ndim == 1 else bwd), st

    def rows_cone(self, mu, y, geom, ray_idx, threads=None, cap=64.0):
        """Both at once (each row walked once): (b [n, C], x [nt, C], status).
        Also sets the crossings' conditioning (``oracle_walk`` in oracle.c):
        ``last_kf`` [n, C, 2] per ray, sum of |mu jump| w kappa / sin over its
        crossings, and ``last_kb`` [nt, C, 2] per tet, sum over the rays
        crossing or touching it of |y| (w kappa / sin)_in + |y| (w kappa /
        sin)_out; [..., 0] with 1 / sin capped at ``cap``, [..., 1] uncapped;
        w = distance from the source + mesh radius, kappa = the crossed face's
        shape factor (sum of squared edges / (2 |n|))."""
        return self._run(mu, y, geom, ray_idx, None, None, threads, cap)

    def trace_rays(self, S, P, max_visits=512, threads=None):
        """Visit sequences of explicit rays: (tet [n, max_visits] int32, a_ij
        [n, max_visits], count [n], status [n]); tets in walk order (rays not
        walked: the brute-force row sorted by entry parameter).  Sets
        ``last_cond`` [n, max_visits, 2]: each visit's (L + R) kappa / sin
        summed over its two crossings (1 / sin capped at 64, uncapped), the
        scale of its chord's rounding error (see ``rows_cone``)."""
        s, sp = _d(S)
        p, pp = _d(P)
        n = s.shape[0]
        tet = np.full((n, max_visits), -1, dtype=np.int32)
        ln = np.zeros((n, max_visits))
        cnt = np.empty(n, dtype=np.int64)
        st = np.empty(n, dtype=np.int8)
        cond = np.zeros((n, max_visits, 2))
        self.last_cond = cond
        _check(lib().oracle_walk_trace(self._h, sp, pp, n, max_visits, tet.ctypes.data_as(_c_ip),
                                       ln.ctypes.data_as(_c_dp), cond.ctypes.data_as(_c_dp),
                                       cnt.ctypes.data_as(_c_lp),
                                       st.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                       threads or default_threads()), "oracle_walk_trace")
        return tet, ln, cnt, st

    def rows_rays(self, mu, y, S, P, threads=None, cap=64.0):
        """``rows_cone`` for explicit rays S, P [n, 3]."""
        return self._run(mu, y, None, None, S, P, threads, cap)

    def forward_rays(self, mu, S, P, threads=None):
        fwd, _, st = self._run(mu, None, None, None, S, P, threads, cond=False)
        return (fwd[:, 0] if np.asarray(mu).ndim == 1 else fwd), st

    def backward_rays(self, y, S, P, threads=None):
        _, bwd, st = self._run(None, y, None, None, S, P, threads, cond=False)
        return (bwd[:, 0] if np.asarray(y).ndim == 1 else bwd), st


def mt_forward_rays(verts, tets, mu, S, P, precision="f64", max_steps=100000):
    """The paper's own walk (Alg. 1-2, mt.c) for explicit rays, in single
    ("f32") or double ("f64") arithmetic: (sums [n], status [n] int8:
    0 done, 1 halted, 2 step limit).  Single-threaded."""
    v, vp = _d(verts)
    t, tp = _i(tets)
    m, mp = _d(np.asarray(mu, dtype=np.float64).reshape(-1))
    s, sp = _d(S)
    p, pp = _d(P)
    n = s.shape[0]
    out = np.zeros(n)
    status = np.zeros(n, np.int8)
    _check(lib().oracle_mt_forward_rays(vp, v.shape[0], tp, t.shape[0], mp, sp, pp, n,
                                        4 if precision == "f32" else 8, int(max_steps),
                                        out.ctypes.data_as(_c_dp),
                                        status.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))),
           "oracle_mt_forward_rays")
    return out, status


def trace_rays(verts, tets, S, P, max_visits=1024, threads=None):
    """Row j of A per ray: (tets, t_lo, t_hi, count, margin, planar).

    tets[j, :count[j]] are the tets with a_ij > 0 sorted by entry parameter;
    margin[j] is the smallest |t_hi - t_lo| * |P - S| over all tets (small =
    the ray grazes an edge or vertex); planar[j] = ray lies in a face plane."""
    v, vp, t, tp = _mesh(verts, tets)
    s, sp = _d(S)
    p, pp = _d(P)
    n = s.shape[0]
    tt = np.full((n, max_visits), -1, np.int32)
    lo = np.zeros((n, max_visits))
    hi = np.zeros((n, max_visits))
    cnt = np.zeros(n, np.int64)
    mg = np.zeros(n)
    pl = np.zeros(n, np.int32)
    _check(lib().oracle_trace_rays(vp, v.shape[0], tp, t.shape[0], sp, pp, n, max_visits,
                                   tt.ctypes.data_as(_c_ip), lo.ctypes.data_as(_c_dp),
                                   hi.ctypes.data_as(_c_dp), cnt.ctypes.data_as(_c_lp),
                                   mg.ctypes.data_as(_c_dp), pl.ctypes.data_as(_c_ip),
                                   threads or default_threads()),
           "oracle_trace_rays")
    return tt, lo, hi, cnt, mg, pl.astype(bool)
