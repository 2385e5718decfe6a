"""Pins for the CPU oracle against facts fixed by the mathematics (no GPU).

The oracle is the plain definition of Eq. 1-3 (brute-force clipping).  It is
checked here against: hand-derived chords (golden file), the closed-form chord
through the cube and through a cell-aligned sub-box, the exact number of
pieces a ray is cut into by the unjittered Kuhn arrangement, exact rational
entry/exit parameters obtained by a different construction (barycentric
crossing points from edge sides), the adjoint identity, invariance under tet
vertex order, and one-sided limits for rays lying in a face plane.
"""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import workloads as W
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _chord_from_interval(iv, S, P):
    if iv is None:
        return 0.0
    d = np.asarray(P, float) - np.asarray(S, float)
    return float(iv[1] - iv[0]) * math.sqrt(float(d @ d))


def test_golden_single_tet(oracle_lib):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    rows = []
    with open(os.path.join(GOLDEN, "single_tet_chords.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    assert len(rows) >= 8
    for r in rows:
        S, P, want = np.array(r[0:3]), np.array(r[3:6]), r[6]
        a, lo, hi = oracle_lib.tet_chord(V, S, P)
        assert abs(a - want) <= 1e-15 * max(1.0, want), (r, a)
        # vertex order / orientation must not matter
        a2, _, _ = oracle_lib.tet_chord(V[[1, 0, 2, 3]], S, P)
        assert abs(a2 - a) <= 1e-15


def _cube_chord(S, P):
    return _chord_from_interval(exact.cube_interval(S, P), S, P)


def test_cube_chord_constant_mu(oracle_lib):
    """mu = 1: b_j is the chord of the half-line through [-1,1]^3 (closed form)."""
    w = W.config1()
    rng = np.random.default_rng(5)
    idx = rng.choice(w.geom.nrays, size=600, replace=False)
    S, P = oracle_lib.cone_rays(w.geom, idx)
    b = oracle_lib.forward_cone(w.verts, w.tets, np.ones(w.tets.shape[0]), w.geom, idx)
    want = np.array([_cube_chord(S[k], P[k]) for k in range(idx.size)])
    # planar rays double count under the closed measure: use one-sided limits
    _, _, _, _, _, planar = oracle_lib.trace_rays(w.verts, w.tets, S, P, max_visits=4)
    ok = ~planar
    assert ok.sum() > 500
    assert np.all(np.abs(b[ok] - want[ok]) <= 1e-12 * np.maximum(want[ok], 1e-3))
    assert (want > 0).sum() > 300 and (want == 0).sum() > 10


def test_subbox_chord(oracle_lib):
    """mu = 1 on the cells with x < 0: closed-form chord of [-1,0]x[-1,1]^2."""
    w = W.config1()
    cen = W.tet_centroids(w.verts, w.tets)
    mu = (cen[:, 0] < 0).astype(float)
    rng = np.random.default_rng(6)
    idx = rng.choice(w.geom.nrays, size=400, replace=False)
    S, P = oracle_lib.cone_rays(w.geom, idx)
    b = oracle_lib.forward_cone(w.verts, w.tets, mu, w.geom, idx)
    _, _, _, _, _, planar = oracle_lib.trace_rays(w.verts, w.tets, S, P, max_visits=4)
    for k in np.nonzero(~planar)[0]:
        iv = exact.box_interval(S[k], P[k], (-1, -1, -1), (0, 1, 1))
        want = _chord_from_interval(iv, S[k], P[k])
        assert abs(b[k] - want) <= 1e-12 * max(want, 1e-3)


def test_kuhn_piece_counts(oracle_lib):
    """Unjittered Kuhn 8^3: pieces per ray = 1 + distinct plane crossings."""
    w = W.config1()
    rng = np.random.default_rng(7)
    idx = rng.choice(w.geom.nrays, size=300, replace=False)
    S, P = oracle_lib.cone_rays(w.geom, idx)
    tets, lo, hi, cnt, margin, planar = oracle_lib.trace_rays(w.verts, w.tets, S, P)
    checked = 0
    for k in range(idx.size):
        want, inplane = exact.kuhn_crossings(8, S[k], P[k])
        if inplane:
            assert planar[k]
            continue
        if margin[k] < 1e-9:
            continue  # grazes an edge or vertex: zero-length pieces are ambiguous
        assert cnt[k] == want, (k, cnt[k], want)
        checked += 1
    assert checked > 250


def test_exact_intervals_jittered(oracle_lib):
    """Cyrus-Beck intervals equal exact barycentric-crossing intervals."""
    rng = W.rng_for(1, 77)
    verts, tets = W.kuhn_cube(3)
    verts = W.jitter_interior(verts, tets, 3, rng)
    S, T = W.random_rays_through_box(40, np.random.default_rng(8))
    n_hit = 0
    for k in range(S.shape[0]):
        for i in range(tets.shape[0]):
            V = verts[tets[i]]
            a, lo, hi = oracle_lib.tet_chord(V, S[k], T[k])
            iv = exact.plucker_interval(V, S[k], T[k])
            if iv is None or iv[1] <= 0:
                assert a == 0.0 or a < 1e-12
                continue
            t0 = max(iv[0], Fr(0))
            want = _chord_from_interval((t0, iv[1]), S[k], T[k])
            assert abs(a - want) <= 1e-12 * max(want, 1e-6) + 1e-14, (k, i, a, want)
            n_hit += 1
    assert n_hit > 100


def test_sum_invariant_mapped_meshes(oracle_lib):
    """sum_i a_ij = hull chord on jittered and cubic-mapped meshes."""
    rng = np.random.default_rng(9)
    S, T = W.random_rays_through_box(60, rng)
    for verts, tets in (
        (W.cubic_map(W.kuhn_cube(6)[0]), W.kuhn_cube(6)[1]),
        (W.jitter_interior(*W.kuhn_cube(6), 6, W.rng_for(1, 5)), W.kuhn_cube(6)[1]),
    ):
        b = oracle_lib.forward_rays(verts, tets, np.ones(tets.shape[0]), S, T)
        want = np.array([_cube_chord(S[k], T[k]) for k in range(S.shape[0])])
        assert np.all(np.abs(b - want) <= 1e-12 * np.maximum(want, 1e-3))


def test_adjoint_identity(oracle_lib):
    """<A x, y> = <x, A^T y> with the forward and backward loops run separately."""
    w = W.config1()
    rng = np.random.default_rng(10)
    idx = rng.choice(w.geom.nrays, size=500, replace=False)
    S, P = oracle_lib.cone_rays(w.geom, idx)
    x = rng.uniform(-1, 1, size=w.tets.shape[0])
    y = rng.uniform(-1, 1, size=idx.size)
    Ax = oracle_lib.forward_rays(w.verts, w.tets, x, S, P)
    Aty = oracle_lib.backward_rays(w.verts, w.tets, y, S, P)
    scale = oracle_lib.forward_rays(w.verts, w.tets, np.abs(x), S, P) @ np.abs(y)
    assert abs(Ax @ y - x @ Aty) <= 1e-12 * scale
    # channels: C = 3 equals three separate C = 1 calls
    X3 = rng.uniform(size=(w.tets.shape[0], 3))
    B3 = oracle_lib.forward_rays(w.verts, w.tets, X3, S, P)
    for c in range(3):
        assert np.allclose(B3[:, c], oracle_lib.forward_rays(w.verts, w.tets, X3[:, c], S, P),
                           rtol=0, atol=1e-13)


def test_cone_backward_matches_rays(oracle_lib):
    w = W.config1(det=8, nangles=3)
    rng = np.random.default_rng(11)
    y = rng.uniform(size=w.geom.nrays)
    S, P = oracle_lib.cone_rays(w.geom)
    a = oracle_lib.backward_cone(w.verts, w.tets, y, w.geom)
    b = oracle_lib.backward_rays(w.verts, w.tets, y, S, P)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-15)
    sub = np.array([0, 17, 1000, 3071])
    c = oracle_lib.backward_cone_subset(w.verts, w.tets, y, w.geom, sub)
    assert np.allclose(c, a[sub], rtol=1e-13, atol=1e-15)


def test_cone_ray_convention(oracle_lib):
    """Pixel centres follow the stated convention (angle 0 and 90 degrees)."""
    g = W.ConeBeam(4.0, 8.0, 4, 2, 0.5, 0.25, np.array([0.0, np.pi / 2]))
    S, P = oracle_lib.cone_rays(g)
    assert np.allclose(S[0], [4, 0, 0])
    # a=0, iv=0, iu=0: u = (0 - 1.5)*0.5 = -0.75, v = (0 - 0.5)*0.25 = -0.125
    assert np.allclose(P[0], [-4, -0.75, -0.125])
    # j = 7: a=0, iv=1, iu=3: u = 0.75, v = 0.125
    assert np.allclose(P[7], [-4, 0.75, 0.125])
    # j = 15: a=1 (90 deg), iv=1, iu=3: C = (0,-4,0), U = (-1,0,0)
    assert np.allclose(P[15], [-0.75, -4, 0.125], atol=1e-14)


def test_planar_rays_one_sided(oracle_lib):
    """Rays inside a face plane: the two one-sided limits each sum to the chord
    for mu = 1, while the closed measure counts the shared face twice."""
    verts, tets = W.kuhn_cube(4)
    # the plane y = z is an arrangement plane; this ray lies in it
    S = np.array([[4.0, 0.1, 0.1], [4.0, 0.0, 0.0]])
    P = np.array([[-4.0, 0.3, 0.3], [-4.0, 0.5, 0.5]])
    one = np.ones(tets.shape[0])
    closed = oracle_lib.forward_rays(verts, tets, one, S, P)
    wdir = np.array([[0.0, 1.0, -1.0], [0.0, 1.0, -1.0]]) + 1e-3 * np.array([[0.3, 0.1, 0.2]] * 2)
    plus = oracle_lib.forward_rays(verts, tets, one, S, P, side=wdir)
    minus = oracle_lib.forward_rays(verts, tets, one, S, P, side=-wdir)
    chord = np.array([_cube_chord(S[k], P[k]) for k in range(2)])
    assert np.allclose(plus, chord, rtol=1e-12)
    assert np.allclose(minus, chord, rtol=1e-12)
    assert np.all(closed > chord * 1.5)
    _, _, _, _, _, planar = oracle_lib.trace_rays(verts, tets, S, P)
    assert planar.all()


def test_miss_is_zero(oracle_lib):
    verts, tets = W.kuhn_cube(2)
    S = np.array([[4.0, 0, 2.5], [0, 0, 5.0]])
    P = np.array([[-4.0, 0, 2.5], [0, 3.0, 5.0]])
    b = oracle_lib.forward_rays(verts, tets, np.ones(tets.shape[0]), S, P)
    assert np.all(b == 0.0)


# Plausible mistakes planted in a compiled copy of oracle.c's clipper: each must
# fail the golden chords or the closed-form cube chord above.
PLANTED = [
    ("exit parameter keeps the largest face crossing", "            if (t < h) h = t;",
     "            if (t > h || h == INFINITY) h = t;"),
    ("face normals oriented inwards",
     "if (side > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }",
     "if (side < 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }"),
    ("the whole line instead of the half-line t >= 0", "    double l = t0, h = t1;",
     "    double l = -INFINITY, h = t1;"),
    ("chord in units of t instead of length",
     "    return hi > lo ? (hi - lo) * sqrt(dot3(d, d)) : 0.0;",
     "    return hi > lo ? (hi - lo) : 0.0;"),
]


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "single_tet_chords.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def _clipper_copy_ok(tmp_path, src):
    """Compile `src` (a copy of oracle.c); True if its chords match the golden
    file and its mu = 1 sums on a jittered 4^3 mesh the cube chord."""
    import ctypes
    import subprocess
    (tmp_path / "oracle.c").write_text(src)
    lib = str(tmp_path / "libclip.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-o", lib, str(tmp_path / "oracle.c"), "-lm"], check=True)
    L = ctypes.CDLL(lib)
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_tet_chord.restype = ctypes.c_double
    L.oracle_tet_chord.argtypes = [dp, dp, dp, dp, dp]
    L.oracle_forward_rays.restype = ctypes.c_int
    L.oracle_forward_rays.argtypes = [dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.c_int64, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int64,
                                      dp, ctypes.c_int]
    V = np.ascontiguousarray([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    for r in _golden_rows():
        S = np.ascontiguousarray(r[0:3], dtype=np.float64)
        P = np.ascontiguousarray(r[3:6], dtype=np.float64)
        a = L.oracle_tet_chord(V.ctypes.data_as(dp), S.ctypes.data_as(dp), P.ctypes.data_as(dp),
                               ctypes.byref(lo), ctypes.byref(hi))
        if not abs(a - r[6]) <= 1e-15 * max(1.0, r[6]):
            return False
    verts, tets = W.kuhn_cube(4)
    verts = np.ascontiguousarray(W.jitter_interior(verts, tets, 4, W.rng_for(9, 2)))
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    S, P = W.random_rays_through_box(300, np.random.default_rng(13))
    S, P = np.ascontiguousarray(S), np.ascontiguousarray(P)
    ones = np.ones(tets.shape[0])
    out = np.zeros(S.shape[0])
    rc = L.oracle_forward_rays(verts.ctypes.data_as(dp), verts.shape[0],
                               tets.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tets.shape[0],
                               ones.ctypes.data_as(dp), 1, S.ctypes.data_as(dp),
                               P.ctypes.data_as(dp), None, S.shape[0], out.ctypes.data_as(dp), 4)
    want = np.array([_cube_chord(S[k], P[k]) for k in range(S.shape[0])])
    return rc == 0 and bool(np.all(np.abs(out - want) <= 1e-12 * np.maximum(want, 1.0)))


def _oracle_source():
    return open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "oracle.c")).read()


def test_clipper_copy_harness_passes_unchanged_source(tmp_path):
    assert _clipper_copy_ok(tmp_path, _oracle_source())


@pytest.mark.parametrize("what,old,new", PLANTED, ids=[p[0] for p in PLANTED])
def test_pins_catch_planted_clipper_mistakes(tmp_path, what, old, new):
    src = _oracle_source()
    assert src.count(old) == 1
    assert not _clipper_copy_ok(tmp_path, src.replace(old, new)), what
