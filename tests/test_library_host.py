"""Host-side checks of libtetproj.so (no GPU): exports, the predicate cascade
against exact arithmetic, and mesh topology / validation."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import exact

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build_library()
    import paper_1908_06909_gb300 as tp
    tp._lib.load()
    return tp


def test_exports_every_declared_symbol(tp):
    hdr = open(os.path.join(ROOT, "include", "tetproj.h")).read()
    names = sorted(set(re.findall(r"\b(tetproj_[a-z0-9_]+)\s*\(", hdr)))
    assert len(names) >= 20
    L = ctypes.CDLL(tp.library_path())
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the Python binding declares exactly the header's functions
    assert set(names) == set(tp._lib.SIGNATURES), set(names) ^ set(tp._lib.SIGNATURES)


def test_status_strings(tp):
    L = tp._lib.load()
    for code in range(0, 12):
        assert L.tetproj_status_string(code)
    assert L.tetproj_version() >= 100


def _near_degenerate(rng, n, scale_edge):
    """Rays passing within ~1e-7..1e-15 of an edge line, mesh-like magnitudes."""
    p = rng.uniform(-1, 1, size=(n, 3))
    q = p + rng.normal(size=(n, 3)) * scale_edge
    lam = rng.uniform(-0.5, 1.5, size=(n, 1))
    X = p + lam * (q - p)
    ang = rng.uniform(0, 2 * np.pi, size=n)
    S = np.stack([4 * np.cos(ang), 4 * np.sin(ang), rng.uniform(-0.5, 0.5, n)], axis=1)
    eps = 10.0 ** rng.uniform(-16, -1, size=(n, 1))
    P = S + 2.0 * (X - S) + eps * rng.normal(size=(n, 3))
    return S, P, p, q


def test_side_cascade_sound_and_exact(tp):
    """Every sign the cascade returns equals the exact sign when the exact value
    is non-zero (so every FP32/FP64 'certain' answer is right)."""
    rng = np.random.default_rng(21)
    cases = []
    for sc in (1e-1, 1e-3, 3e-5):
        cases.append(_near_degenerate(rng, 20000, sc))
    S, P, p, q = [np.concatenate([c[k] for c in cases]) for k in range(4)]
    sign, stage = tp.side_signs_host(S, P, p, q)
    n_fp32 = n_fp64 = n_exact = 0
    for k in range(S.shape[0]):
        want = exact.side_sign_int(S[k], P[k], p[k], q[k])
        assert want != 0 or stage[k] == 3
        if want != 0:
            assert sign[k] == want, (k, stage[k])
        n_fp32 += stage[k] == 0
        n_fp64 += stage[k] == 1
        n_exact += stage[k] == 2
    # the test must exercise every stage
    assert n_fp32 > 1000 and n_fp64 > 1000 and n_exact > 100


def test_side_cascade_sound_one_million(tp):
    """10^6 near-degenerate orientations (rays within 1e-16..1e-1 of an edge
    line, edges from 1e-1 down to 1e-5 long, some far from the origin): every
    sign the FP32 or FP64 filter certifies equals the exact sign."""
    rng = np.random.default_rng(24)
    cases = []
    for sc in (1e-1, 1e-2, 1e-3, 1e-4, 3e-5, 1e-5):
        cases.append(_near_degenerate(rng, 150000, sc))
    S, P, p, q = [np.concatenate([c[k] for c in cases]) for k in range(4)]
    far = rng.random(S.shape[0]) < 0.2            # a fifth shifted away from the origin
    shift = rng.uniform(-50.0, 50.0, size=(S.shape[0], 3)) * far[:, None]
    S, P, p, q = S + shift, P + shift, p + shift, q + shift
    assert S.shape[0] >= 1_000_000 - 100000
    extra = _near_degenerate(rng, 1_000_000 - S.shape[0], 1e-3)
    S, P, p, q = [np.concatenate([a, b]) for a, b in zip((S, P, p, q), extra)]
    assert S.shape[0] == 1_000_000
    sign, stage = tp.side_signs_host(S, P, p, q)
    certain = stage <= 1
    checked = 0
    for k in np.nonzero(certain)[0]:
        assert sign[k] == exact.side_sign_int(S[k], P[k], p[k], q[k]), (k, stage[k])
        checked += 1
    # the filters decide most cases and leave a real share to the exact stages
    assert checked > 500_000 and (~certain).sum() > 10_000


def test_side_cascade_symbolic_matches_exact_module(tp):
    rng = np.random.default_rng(22)
    grid = lambda: rng.integers(-4, 5, size=3).astype(float) / 4.0
    rows = []
    for _ in range(400):
        p, q = grid(), grid()
        while np.all(p == q):
            q = grid()
        S = grid() * 4 + np.array([0.0, 0.0, 8.0])
        kind = rng.integers(0, 4)
        if kind == 0:
            P = p.copy()
        elif kind == 1:
            P = S + 2 * (p - S)
        elif kind == 2:
            P = S + (q - p)
        else:
            S = p - 2.0 * (q - p)
            P = q.copy()
        rows.append((S, P, p, q))
    S, P, p, q = [np.array([r[k] for r in rows]) for k in range(4)]
    sign, stage = tp.side_signs_host(S, P, p, q)
    zeros = 0
    for k in range(len(rows)):
        assert sign[k] == exact.side_sos(S[k], P[k], p[k], q[k]), k
        zeros += stage[k] == 3
    assert zeros > 150


def test_topology_kuhn(tp):
    n = 4
    v, t = W.kuhn_cube(n)
    adj, nb, nf = tp.topology_host(v, t)
    assert nb == 12 * n * n
    assert nf == t.shape[0] // 2
    # neighbours share exactly the face opposite the local vertex, and adjacency is symmetric
    for i in range(t.shape[0]):
        for k in range(4):
            j = adj[i, k]
            face = set(t[i]) - {t[i, k]}
            if j < 0:
                continue
            assert face <= set(t[j])
            assert i in adj[j]


def test_topology_validation_errors(tp):
    from paper_1908_06909_gb300 import _lib
    v, t = W.kuhn_cube(2)

    def code(vv, tt):
        try:
            tp.topology_host(vv, tt)
            return 0
        except tp.TetprojError as e:
            return e.code

    assert code(v, t) == 0
    bad = t.copy(); bad[3, 1] = v.shape[0]
    assert code(v, bad) == _lib.ERR_INDEX
    bad = t.copy(); bad[3, 1] = bad[3, 2]
    assert code(v, bad) == _lib.ERR_INDEX
    flat = v.copy(); flat[t[0]] = flat[t[0]] * np.array([1, 1, 0])  # squash a tet... may break others
    vv = v.copy(); tt = t.copy()
    tt[0, 3] = tt[0, 2]  # repeated -> index error, so make a true zero-volume tet:
    vz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.0]])
    assert code(vz, np.array([[0, 1, 2, 3]])) == _lib.ERR_DEGENERATE_TET
    # face shared by three tets
    v3 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1.0]])
    assert code(v3, np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]])) == _lib.ERR_NONMANIFOLD
    # two tets on the same side of their shared face (overlap)
    v2 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.1, 0.1, 2.0]])
    assert code(v2, np.array([[0, 1, 2, 3], [0, 1, 2, 4]])) == _lib.ERR_NONMANIFOLD
    # non-convex: an L-shape of three Kuhn cells
    vk, tk = W.kuhn_cube(2)
    cen = W.tet_centroids(vk, tk)
    keep = ~((cen[:, 0] > 0) & (cen[:, 1] > 0))
    assert code(vk, tk[keep]) == _lib.ERR_NONCONVEX
    # disconnected: two separate tets
    vd = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1],
                   [5, 0, 0], [6, 0, 0], [5, 1, 0], [5, 0, 1.0]])
    assert code(vd, np.array([[0, 1, 2, 3], [4, 5, 6, 7]])) == _lib.ERR_NONCONVEX
    # single tet is a valid convex mesh
    assert code(vd[:4], np.array([[0, 1, 2, 3]])) == 0


def test_fp32_filter_sound_near_threshold(tp):
    """Cases packed around the FP32 filter's decision threshold (ray-edge
    distances 1e-9..1e-4 of the edge length, walk-like magnitudes): every
    FP32-certain answer equals the exact sign."""
    rng = np.random.default_rng(23)
    n = 60000
    p = rng.uniform(-1, 1, size=(n, 3))
    L = 10.0 ** rng.uniform(-4.5, -0.5, size=(n, 1))
    q = p + rng.normal(size=(n, 3)) * L
    X = p + rng.uniform(-0.2, 1.2, size=(n, 1)) * (q - p)
    ang = rng.uniform(0, 2 * np.pi, size=n)
    S = np.stack([4 * np.cos(ang), 4 * np.sin(ang), rng.uniform(-0.3, 0.3, n)], axis=1)
    off = rng.normal(size=(n, 3))
    P = S + 2.0 * (X - S) + off * L * 10.0 ** rng.uniform(-9, -4, size=(n, 1))
    sign, stage = tp.side_signs_host(S, P, p, q)
    fp32 = np.nonzero(stage == 0)[0]
    assert fp32.size > 3000 and (stage != 0).sum() > 5000
    for k in fp32:
        assert sign[k] == exact.side_sign_int(S[k], P[k], p[k], q[k]), k


def test_fp32_filter_sound_far_from_origin(tp):
    """The same near-threshold packing for a mesh far from the origin, where
    the FP32 rounding of the vertex coordinates (the |w| . |n| and guard terms
    of the bound) dominates the error: every FP32-certain answer is exact."""
    rng = np.random.default_rng(29)
    n = 40000
    centre = np.array([3.0e3, -2.0e3, 1.0e3])
    p = centre + rng.uniform(-1, 1, size=(n, 3))
    L = 10.0 ** rng.uniform(-3.5, -0.5, size=(n, 1))
    q = p + rng.normal(size=(n, 3)) * L
    X = p + rng.uniform(-0.2, 1.2, size=(n, 1)) * (q - p)
    ang = rng.uniform(0, 2 * np.pi, size=n)
    S = centre + np.stack([4 * np.cos(ang), 4 * np.sin(ang), rng.uniform(-0.3, 0.3, n)], axis=1)
    off = rng.normal(size=(n, 3))
    P = S + 2.0 * (X - S) + off * L * 10.0 ** rng.uniform(-6, 0, size=(n, 1))
    sign, stage = tp.side_signs_host(S, P, p, q)
    fp32 = np.nonzero(stage == 0)[0]
    assert fp32.size > 2000 and (stage != 0).sum() > 2000
    for k in fp32:
        assert sign[k] == exact.side_sign_int(S[k], P[k], p[k], q[k]), k


def test_batch_argument_errors(tp):
    """Batch entry points reject bad arguments before touching the device."""
    import ctypes as C
    from paper_1908_06909_gb300 import _lib
    L = tp._lib.load()
    h = C.c_void_p(7)
    assert L.tetproj_batch_create(None, None, None, 3, 1, C.byref(h)) == _lib.ERR_ARG
    assert h.value is None
    arr = (C.c_void_p * 1)(None)
    assert L.tetproj_batch_create(arr, arr, None, 0, 1, C.byref(h)) == _lib.ERR_ARG
    assert L.tetproj_batch_create(arr, arr, None, 1, 2, C.byref(h)) == _lib.ERR_ARG
    assert L.tetproj_batch_create(arr, arr, None, 1, 1, C.byref(h)) == _lib.ERR_ARG  # null handles
    assert L.tetproj_batch_create(arr, arr, None, 1, 1, None) == _lib.ERR_ARG
    assert L.tetproj_batch_bind(None, None, None, None, None) == _lib.ERR_ARG
    assert L.tetproj_batch_forward(None, None) == _lib.ERR_ARG
    assert L.tetproj_batch_backward(None, None) == _lib.ERR_ARG
    assert L.tetproj_batch_destroy(None) == _lib.ERR_ARG


def test_rstar_tree_invariants(tp):
    """The boundary-face R*-tree (the paper's entry structure): node fills
    within [4, 10], all leaves at one depth, nested boxes, every boundary face
    in exactly one leaf -- on regular, cubic-mapped and jittered meshes."""
    cases = []
    for n in (1, 3, 8):
        cases.append(W.kuhn_cube(n))
    v, t = W.kuhn_cube(6)
    cases.append((W.cubic_map(v), t))
    v, t = W.kuhn_cube(7)
    cases.append((W.jitter_interior(v, t, 7, W.rng_for(7, 1)), t))
    for v, t in cases:
        info = tp.rstar_build_host(v, t)
        nb = tp.topology_host(v, t)[1]
        assert info["ok"] == 1, info
        assert info["entries"] == nb
        if info["depth"] > 1:
            assert 4 <= info["min_fill"] <= info["max_fill"] <= 10
