"""Pins of the oracle walker (oracle.Walker) -- CPU only.

The walker finds the tets a ray crosses by walking face adjacency that it
builds itself, and clips each with the brute-force clipper's own code, so it
must give the brute-force rows of A exactly (summation order aside).  Pinned
here against things outside the walker: the brute-force clipper (every tet
tested against every ray), the closed-form chord of the cube (mu = 1), the
per-ray tet counts of the brute-force trace, and mesh errors it must reject.
It is also checked that the walk itself is what produces the values (most
rays walked, not handed to the brute-force fallback).
"""
import numpy as np
import pytest

import oracle
import workloads as W


def cube_chord(S, P):
    """|{t >= 0 : S + t (P - S) in [-1, 1]^3}| * |P - S| (slab method)."""
    d = P - S
    t0 = np.zeros(S.shape[0])
    t1 = np.full(S.shape[0], np.inf)
    for k in range(3):
        with np.errstate(divide="ignore", invalid="ignore"):
            a = (-1.0 - S[:, k]) / d[:, k]
            b = (1.0 - S[:, k]) / d[:, k]
        lo = np.where(d[:, k] == 0, np.where(np.abs(S[:, k]) <= 1, -np.inf, np.inf), np.minimum(a, b))
        hi = np.where(d[:, k] == 0, np.where(np.abs(S[:, k]) <= 1, np.inf, -np.inf), np.maximum(a, b))
        t0 = np.maximum(t0, lo)
        t1 = np.minimum(t1, hi)
    return np.maximum(0.0, t1 - t0) * np.linalg.norm(d, axis=1)


def small_meshes():
    c2 = W.config2(n_cells=8, det=24, pitch=0.25, nangles=12)
    c3 = W.config3(n_cells=8, det=24, pitch=0.25, nangles=12, n_adversarial=0)
    c5 = W.config5_problem(3, 6, 20, 10)
    return {"jittered": c2, "cubic": c3, "c5like": c5}


@pytest.fixture(scope="module")
def meshes():
    return small_meshes()


def test_config1_all_rays_equal_brute_force():
    w = W.config1()
    wk = oracle.Walker(w.verts, w.tets)
    got, st = wk.forward_cone(w.mu, w.geom)
    want = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom)
    scale = oracle.forward_cone(w.verts, w.tets, np.abs(w.mu), w.geom)
    assert np.all(np.abs(got - want) <= 1e-14 * scale)
    # the unjittered grid has many rays through edges: those take the fallback
    assert (st == 0).mean() > 0.9
    # rays reported in a face plane are planar by the brute-force trace too
    S, P = oracle.cone_rays(w.geom)
    planar = oracle.trace_rays(w.verts, w.tets, S, P, max_visits=2)[5]
    assert np.all(planar[st == 2])


@pytest.mark.parametrize("name", ["jittered", "cubic", "c5like"])
def test_forward_and_backward_equal_brute_force(meshes, name):
    w = meshes[name]
    wk = oracle.Walker(w.verts, w.tets)
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(w.geom.nrays, 2000, replace=False))
    mu = np.asarray(w.mu)
    got, st = wk.forward_cone(mu, w.geom, idx)
    want = oracle.forward_cone(w.verts, w.tets, mu, w.geom, idx)
    scale = oracle.forward_cone(w.verts, w.tets, np.abs(mu), w.geom, idx)
    assert np.all(np.abs(got - want) <= 1e-14 * scale + 1e-300)
    assert (st == 0).mean() > 0.9, np.bincount(st)
    C = 1 if mu.ndim == 1 else mu.shape[1]
    y = rng.uniform(-1.0, 1.0, size=(idx.size, C)).squeeze()
    x, _ = wk.backward_cone(y, w.geom, idx)
    S, P = oracle.cone_rays(w.geom, idx)
    xb = oracle.backward_rays(w.verts, w.tets, y, S, P)
    xs = oracle.backward_rays(w.verts, w.tets, np.abs(y), S, P)
    assert np.all(np.abs(x - xb) <= 1e-14 * xs + 1e-300)
    # per-tet crossing counts = the brute-force trace's rows
    tr_tet, _, _, tr_count = oracle.trace_rays(w.verts, w.tets, S, P, max_visits=512)[:4]
    assert tr_count.max() <= 512
    cnt = np.zeros(w.tets.shape[0], np.int64)
    for k in range(idx.size):
        np.add.at(cnt, tr_tet[k, :tr_count[k]], 1)
    assert np.array_equal(wk.last_count, cnt)


def test_explicit_rays_and_cube_chord(meshes):
    w = meshes["jittered"]
    wk = oracle.Walker(w.verts, w.tets)
    S, P = W.random_rays_through_box(3000, np.random.default_rng(11))
    ones = np.ones(w.tets.shape[0])
    chord, st = wk.forward_rays(ones, S, P)
    # Sum_i a_ij = the chord of the cube (jitter moves interior vertices only)
    ref = cube_chord(S, P)
    assert np.all(np.abs(chord - ref) <= 1e-12 * np.maximum(ref, 1.0))
    assert (ref > 0).sum() > 1000 and (st[ref > 0] == 0).mean() > 0.95
    mu = np.asarray(w.mu)
    got, _ = wk.forward_rays(mu, S, P)
    want = oracle.forward_rays(w.verts, w.tets, mu, S, P)
    assert np.all(np.abs(got - want) <= 1e-14 * oracle.forward_rays(w.verts, w.tets, np.abs(mu), S, P) + 1e-300)


def test_walk_is_what_produces_the_rows(meshes):
    """The same mesh with its vertex ids and tet order permuted (so the
    adjacency the walker builds, its face buckets and its boundary list all
    change) gives the same values."""
    w = meshes["jittered"]
    rng = np.random.default_rng(3)
    perm_v = rng.permutation(w.verts.shape[0])
    inv = np.empty_like(perm_v)
    inv[perm_v] = np.arange(perm_v.size)
    perm_t = rng.permutation(w.tets.shape[0])
    verts2 = w.verts[perm_v]
    tets2 = inv[w.tets[perm_t]]
    mu2 = np.asarray(w.mu)[perm_t]
    idx = np.arange(0, w.geom.nrays, 5)
    a, _ = oracle.Walker(w.verts, w.tets).forward_cone(w.mu, w.geom, idx)
    b, _ = oracle.Walker(verts2, tets2).forward_cone(mu2, w.geom, idx)
    assert np.all(np.abs(a - b) <= 1e-13 * np.maximum(np.abs(a), 1e-3))


def test_rejects_bad_meshes():
    verts, tets = W.kuhn_cube(2)
    bad = np.concatenate([tets, tets[:1]])  # a tet twice: its faces are shared three times
    with pytest.raises(RuntimeError, match="-3"):
        oracle.Walker(verts, bad)
    bad = tets.copy()
    bad[0, 0] = verts.shape[0]
    with pytest.raises(RuntimeError, match="-4"):
        oracle.Walker(verts, bad)


def test_entries_through_boundary_edges_and_vertices():
    """Rays that enter the mesh exactly through a boundary edge or vertex can
    cross no tet with a boundary face first (the tet they enter may touch the
    boundary only there); the walker must still give the brute-force row, not
    a miss.  Entry points on the x = 1 face: grid vertices, points of grid
    lines, midpoints of the face diagonals; sources at random directions
    outside that face (so no ray lies in a face plane)."""
    verts, tets = W.kuhn_cube(4)
    verts = W.jitter_interior(verts, tets, 4, W.rng_for(9, 1))
    rng = np.random.default_rng(2)
    mu = rng.uniform(0.5, 1.5, tets.shape[0])
    g = np.linspace(-1.0, 1.0, 5)[1:-1]
    E = [(1.0, a, b) for a in g for b in g]
    E += [(1.0, a, z) for a in g for z in rng.uniform(-0.9, 0.9, 3)]
    E += [(1.0, z, a) for a in g for z in rng.uniform(-0.9, 0.9, 3)]
    E += [(1.0, a + 0.25, b + 0.25) for a in g for b in g]
    E = np.array(E)
    u = rng.normal(size=E.shape)
    u[:, 0] = np.abs(u[:, 0]) + 0.5
    S = E + 3.0 * u / np.linalg.norm(u, axis=1, keepdims=True)
    P = E + (E - S)
    wk = oracle.Walker(verts, tets)
    got, st = wk.forward_rays(mu, S, P)
    want = oracle.forward_rays(verts, tets, mu, S, P)
    assert np.all(np.abs(got - want) <= 1e-14 * np.abs(want) + 1e-300)
    assert np.all(want > 0)
    assert np.all(st < 2) and np.any(st == 1)


def test_ray_entering_and_leaving_through_boundary_edges():
    """Problem #5 of the batched workload (jittered Kuhn 21^3), cone ray 35,374
    (angle 0, source (4, 0, 0)): it enters the cube exactly on the boundary
    grid line y = -3/7 of the face x = 1 and leaves on y = -5/7 of x = -1, and
    every tet it crosses with positive length touches the boundary at most in
    an edge.  No tet with a boundary face is crossed, yet the ray is not a
    miss: the brute-force row (sum 0.986 on channel 0)."""
    n, N, na = W.config5_specs()[5]
    w = W.config5_problem(5, n, N, na, channels=4)
    idx = np.array([35372, 35373, 35374, 35375, 35376])
    got, st = oracle.Walker(w.verts, w.tets).forward_cone(w.mu, w.geom, idx)
    want = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom, idx)
    assert np.all(np.abs(got - want) <= 1e-14 * np.abs(want) + 1e-300)
    assert want[2, 0] > 0.9 and st[2] == 1


def test_crossing_conditioning_by_hand():
    """The conditioning sums the parity tests scale their floors by, on the
    corner tet (0,0,0), (1,0,0), (0,1,0), (0,0,1) and the ray from (-2, .1, .2)
    along +x (d = (4, 0, 0)): it enters through x = 0 at t = 1/2 (distance 2
    from the source, sin 1; the face's edges 1, 1, sqrt 2 and |n| = 1 give the
    shape factor (1 + 1 + 2) / 2 = 2) and leaves through x + y + z = 1 at
    x = 0.7, t = 0.675 (distance 2.7, sin 1/sqrt 3; edges sqrt 2, |n| = sqrt 3:
    factor 6 / (2 sqrt 3) = sqrt 3); mesh radius 1.  Per ray
    K = |mu| (2 + 1) 2 / 1 + |mu| (2.7 + 1) sqrt 3 sqrt 3; per tet the same
    with |y|; with 1 / sin capped at 1 the second term's sin factor is 1."""
    verts = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    tets = np.array([[0, 1, 2, 3]])
    S = np.array([[-2.0, 0.1, 0.2]])
    P = S + np.array([[4.0, 0, 0]])
    wk = oracle.Walker(verts, tets)
    r3 = np.sqrt(3.0)
    for cap, g_out in ((64.0, r3), (1.0, 1.0)):
        fwd, bwd, st = wk.rows_rays(np.array([-1.5]), np.array([2.0]), S, P, threads=1, cap=cap)
        assert st[0] == 0 and abs(fwd[0, 0] - (-1.5 * 0.7)) < 1e-15
        want = 6.0 + 3.7 * r3 * g_out
        assert abs(wk.last_kf[0, 0, 0] - 1.5 * want) < 1e-13
        assert abs(wk.last_kf[0, 0, 1] - 1.5 * (6.0 + 3.7 * 3.0)) < 1e-13
        assert abs(wk.last_kb[0, 0, 0] - 2.0 * want) < 1e-13
        assert abs(bwd[0, 0] - 2.0 * 0.7) < 1e-15
    tet, ln, cnt, st = wk.trace_rays(S, P, max_visits=4)
    assert cnt[0] == 1 and tet[0, 0] == 0 and abs(ln[0, 0] - 0.7) < 1e-15
    assert abs(wk.last_cond[0, 0, 1] - (6.0 + 3.7 * 3.0)) < 1e-13


def test_crossing_conditioning_constant_mu(meshes):
    """mu = 1 on a jittered mesh: mu jumps only where the ray enters and leaves
    the cube, so K = 2 (L_in + R) / sin_in + 2 (L_out + R) / sin_out with the
    cube's axis faces (sin = |d_k| / |d| for the face normal to axis k; the
    boundary faces are unjittered right isosceles triangles: shape factor
    (h^2 + h^2 + 2 h^2) / (2 h^2) = 2), L the distance from the source,
    R = 1."""
    w = meshes["jittered"]
    wk = oracle.Walker(w.verts, w.tets)
    S, P = W.random_rays_through_box(2000, np.random.default_rng(12))
    d = P - S
    dn = np.linalg.norm(d, axis=1)
    chord = cube_chord(S, P)
    ok = chord > 1e-3
    _, _, st = wk.rows_rays(np.ones(w.tets.shape[0]), None, S[ok], P[ok])
    K = wk.last_kf[:, 0, 1]
    t_in = np.full(S.shape[0], -np.inf)
    t_out = np.full(S.shape[0], np.inf)
    ax_in = np.zeros(S.shape[0], int)
    ax_out = np.zeros(S.shape[0], int)
    for k in range(3):
        with np.errstate(divide="ignore"):
            a = (-1.0 - S[:, k]) / d[:, k]
            b = (1.0 - S[:, k]) / d[:, k]
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        ax_in = np.where(lo > t_in, k, ax_in)
        t_in = np.maximum(t_in, lo)
        ax_out = np.where(hi < t_out, k, ax_out)
        t_out = np.minimum(t_out, hi)
    r = np.arange(S.shape[0])
    want = 2.0 * ((t_in * dn + 1.0) * dn / np.abs(d[r, ax_in]) +
                  (t_out * dn + 1.0) * dn / np.abs(d[r, ax_out]))[ok]
    keep = st == 0
    assert keep.mean() > 0.95
    assert np.all(np.abs(K[keep] - want[keep]) <= 1e-9 * want[keep])


@pytest.mark.parametrize("name", ["jittered", "cubic"])
def test_trace_equals_brute_force_trace(meshes, name):
    """Visit sequences: the walker's order and a_ij equal the brute-force
    trace (all tets clipped, sorted by entry parameter) on walked rays."""
    w = meshes[name]
    idx = np.sort(np.random.default_rng(8).choice(w.geom.nrays, 1500, replace=False))
    S, P = oracle.cone_rays(w.geom, idx)
    tet, ln, cnt, st = oracle.Walker(w.verts, w.tets).trace_rays(S, P, max_visits=256)
    bt, blo, bhi, bcnt = oracle.trace_rays(w.verts, w.tets, S, P, max_visits=256)[:4]
    # rows not walked also list the tets a ray only touches, with a_ij = 0
    assert np.array_equal((ln > 0).sum(axis=1), bcnt)
    assert np.all(cnt[st == 0] == bcnt[st == 0])
    dl = np.linalg.norm(P - S, axis=1)
    walked = np.nonzero(st == 0)[0]
    assert walked.size > 0.9 * idx.size
    for k in walked:
        n = cnt[k]
        assert np.array_equal(tet[k, :n], bt[k, :n]), k
        assert np.array_equal(ln[k, :n], (bhi[k, :n] - blo[k, :n]) * dl[k])


def test_crossing_conditioning_at_an_edge():
    """A ray entering the corner tet exactly through its edge (0,0,0)-(0,0,1),
    at (0, 0, 1/2), along d = (2, 4, 0) from S = (-1, -2, 1/2): two face planes
    pass through the entry point, x = 0 (sin = 2/|d| = 1/sqrt 5) and y = 0
    (sin 2/sqrt 5), both with shape factor 2; the bound takes the worse,
    1/sin = sqrt 5.  Entry at t = 1/2 (distance sqrt 5), exit through
    x + y + z = 1 at t = 7/12 (distance 7 sqrt 5 / 6, sin 3/sqrt 15, shape
    factor sqrt 3); chord sqrt 5 / 6; mesh radius 1."""
    verts = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    tets = np.array([[0, 1, 2, 3]])
    S = np.array([[-1.0, -2.0, 0.5]])
    P = np.array([[1.0, 2.0, 0.5]])
    wk = oracle.Walker(verts, tets)
    fwd, bwd, st = wk.rows_rays(np.array([1.0]), np.array([1.0]), S, P)
    r5 = np.sqrt(5.0)
    assert st[0] == 1  # the entry is a tie: the row comes from the clipper
    assert abs(fwd[0, 0] - r5 / 6) < 1e-15
    want = (r5 + 1.0) * 2.0 * r5 + (7 * r5 / 6 + 1.0) * np.sqrt(3.0) * np.sqrt(15.0) / 3.0
    assert abs(wk.last_kf[0, 0, 1] - want) < 1e-12 * want
    assert abs(wk.last_kb[0, 0, 1] - want) < 1e-12 * want


# Plausible mistakes planted in a copy of oracle.c: each must fail one of the
# pins above (values equal to the brute-force clipper's, most rays walked).
PLANTED = [
    ("exit through the farthest face plane",
     "if (den[k] > 0.0 && (g < 0 || tf[k] < tf[g])) g = k;",
     "if (den[k] > 0.0 && (g < 0 || tf[k] > tf[g])) g = k;"),
    ("neighbour's tet index off by one",
     "w->adj[f[x].code] = f[x + 1].code >> 2;",
     "w->adj[f[x].code] = (f[x + 1].code >> 2) ^ 1;"),
    ("entry through the last boundary tet instead of the first",
     "if (l < lo) { second = lo; lo = l; hi = h; cur = w->btet[q]; }",
     "if (lo == INFINITY || l > lo) { second = INFINITY; lo = l; hi = h; cur = w->btet[q]; }"),
    ("chord measured from the source instead of the entry",
     "if (wpush(out, cur, (hi - lo) * len, lo, hi)) return -1;",
     "if (wpush(out, cur, hi * len, lo, hi)) return -1;"),
]


def _walk_copy(tmp_path, w, src):
    """Compile `src` (a copy of oracle.c) and walk every 5th cone ray of `w`
    with it: (values equal the clipper's, more than 90% of rays walked)."""
    import ctypes
    import subprocess
    (tmp_path / "oracle.c").write_text(src)
    lib = str(tmp_path / "libcopy.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-o", lib, str(tmp_path / "oracle.c"), "-lm"], check=True)
    L = ctypes.CDLL(lib)
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_walker_create.restype = ctypes.c_void_p
    L.oracle_walker_create.argtypes = [dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    L.oracle_walk.restype = ctypes.c_int
    L.oracle_walk.argtypes = ([ctypes.c_void_p, dp, dp, ctypes.c_int] + [ctypes.c_double] * 2 +
                              [ctypes.c_int64] * 2 + [ctypes.c_double] * 2 +
                              [dp, ctypes.c_int64, ctypes.c_void_p, dp, dp, ctypes.c_int64, dp, dp,
                               ctypes.c_void_p, ctypes.c_double, dp, dp,
                               ctypes.POINTER(ctypes.c_int8), ctypes.c_int])
    L.oracle_walker_destroy.argtypes = [ctypes.c_void_p]
    v = np.ascontiguousarray(w.verts, dtype=np.float64)
    t = np.ascontiguousarray(w.tets, dtype=np.int32)
    st = ctypes.c_int(0)
    h = L.oracle_walker_create(v.ctypes.data_as(dp), v.shape[0],
                               t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), t.shape[0],
                               ctypes.byref(st))
    assert h
    S, P = oracle.cone_rays(w.geom, np.arange(0, w.geom.nrays, 5))
    S, P = np.ascontiguousarray(S), np.ascontiguousarray(P)
    n = S.shape[0]
    mu = np.ascontiguousarray(w.mu, dtype=np.float64)
    out = np.zeros(n)
    status = np.zeros(n, dtype=np.int8)
    rc = L.oracle_walk(h, mu.ctypes.data_as(dp), None, 1, 0.0, 0.0, 0, 0, 0.0, 0.0, None, 0, None,
                       S.ctypes.data_as(dp), P.ctypes.data_as(dp), n, out.ctypes.data_as(dp), None,
                       None, 64.0, None, None, status.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), 4)
    L.oracle_walker_destroy(h)
    want = oracle.forward_rays(w.verts, w.tets, mu, S, P)
    values_ok = rc == 0 and bool(np.all(np.abs(out - want) <= 1e-14 * np.abs(want) + 1e-300))
    return values_ok, bool((status == 0).mean() > 0.9)


def _oracle_source():
    import os
    return open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()


def test_copy_harness_passes_unchanged_source(tmp_path, meshes):
    assert _walk_copy(tmp_path, meshes["jittered"], _oracle_source()) == (True, True)


@pytest.mark.parametrize("what,old,new", PLANTED, ids=[p[0] for p in PLANTED])
def test_pins_catch_planted_mistakes(tmp_path, meshes, what, old, new):
    src = _oracle_source()
    assert src.count(old) == 1
    values_ok, walked_ok = _walk_copy(tmp_path, meshes["jittered"], src.replace(old, new))
    assert not (values_ok and walked_ok), what
