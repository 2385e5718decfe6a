"""Pins for the oracle helpers that the GPU parity tests use as references
(no GPU).

The parity tests take their expected values from the brute-force clipper
except for rays in or near a face plane, where they use:
* ``exact.ray_integral_exact`` (rays near a face plane; exact integers),
* ``oracle.forward_rays_exact_planar`` over ``oracle.forward_rays_range``
  (rays exactly in a face plane: the limit of the symbolically perturbed line),
* ``exact.ray_in_face_plane`` (which of the two a ray gets).
Each is checked here against something other than itself: the clipper (a
different construction, plane equations in FP64), closed-form chords of the
cube and of half-spaces bounded by Kuhn planes, hand-derived partial chords
(tests/golden/single_tet_partial_chords.txt), additivity over parameter
ranges, and constructed in-plane / one-ulp-off / vertex-hitting rays.
Eq. 1-3 fix all of these: a_ij is the length of ray j inside tet i.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _chord(iv, S, P, t0=0.0, t1=math.inf):
    if iv is None:
        return 0.0
    lo = max(float(iv[0]), t0)
    hi = min(float(iv[1]), t1)
    d = np.asarray(P, float) - np.asarray(S, float)
    return max(0.0, hi - lo) * math.sqrt(float(d @ d))


def _exact_chord(iv, S, P):
    if iv is None:
        return 0.0
    d = np.asarray(P, float) - np.asarray(S, float)
    return float(iv[1] - iv[0]) * math.sqrt(float(d @ d))


def _meshes4():
    v, t = W.kuhn_cube(4)
    yield "jittered4", W.jitter_interior(v, t, 4, W.rng_for(2, 41)), t
    yield "cubic4", W.cubic_map(v), t


# ------------------------------------------------------------ ray_integral_exact

@pytest.mark.parametrize("name,verts,tets", list(_meshes4()))
def test_ray_integral_exact_matches_clipper(oracle_lib, name, verts, tets):
    """Generic rays: the exact integer integral equals the FP64 clipper."""
    rng = np.random.default_rng(101)
    S, T = W.random_rays_through_box(40, rng)
    mu = rng.uniform(0.0, 1.0, size=tets.shape[0])
    b = oracle_lib.forward_rays(verts, tets, mu, S, T)
    scale = oracle_lib.forward_rays(verts, tets, np.abs(mu), S, T)
    hits = 0
    for k in range(S.shape[0]):
        e = exact.ray_integral_exact(verts, tets, mu, S[k], T[k])
        # the clipper places each crossing to a few ulps of the coordinates:
        # relative 1e-14 plus the coordinate quantum 16 u R max|mu|
        R = max(np.abs(S[k]).max(), np.abs(T[k]).max(), 1.0)
        assert abs(e - b[k]) <= 1e-14 * scale[k] + 16 * 2.0 ** -53 * R, (name, k, e, b[k])
        hits += e > 0
    assert hits > 20


def test_ray_integral_exact_near_plane_closed_form():
    """mu = 1 on rays one ulp off a Kuhn plane: the integral is the cube chord
    (the rays are not in the plane, so it is unique), and ray_in_face_plane
    tells them apart from the in-plane rays they were made from."""
    verts, tets = W.kuhn_cube(4)
    one = np.ones(tets.shape[0])
    cases = [  # (S, P in plane, index of the coordinate nudged by one ulp)
        ((4.0, 0.1, 0.1), (-4.0, 0.3, 0.3), 2),        # plane y = z
        ((0.5, -4.0, 0.3), (0.5, 4.0, -0.2), 0),       # plane x = 0.5
        ((4.5, 4.0, 0.3), (-3.5, -4.0, -0.1), 1),      # plane x - y = 0.5
        ((0.3, -4.5, -4.0), (-0.1, 3.5, 4.0), 2),      # plane y - z = -0.5
    ]
    for S, P, c in cases:
        S = np.array(S)
        P = np.array(P)
        assert exact.ray_in_face_plane(verts, tets, S, P)
        for direction in (+1.0, -1.0):
            Q = P.copy()
            Q[c] = np.nextafter(Q[c], direction * np.inf)
            assert not exact.ray_in_face_plane(verts, tets, S, Q)
            got = exact.ray_integral_exact(verts, tets, one, S, Q)
            want = _exact_chord(exact.cube_interval(S, Q), S, Q)
            assert want > 1.0
            assert abs(got - want) <= 4e-16 * want, (S, Q, got, want)


def test_ray_integral_exact_raises_on_vertex_and_edge_rays():
    verts, tets = W.kuhn_cube(4)
    mu = np.ones(tets.shape[0])
    S = np.array([4.0, 0.13, 0.21])
    for P in ((0.5, 0.0, -0.5),            # a mesh vertex
              (0.25, 0.0, -0.5),           # midpoint of a cell edge
              (0.25, 0.25, 0.25)):         # midpoint of a cell's main diagonal (a Kuhn edge)
        with pytest.raises(exact.DegenerateRay):
            exact.ray_integral_exact(verts, tets, mu, S, np.array(P))


@pytest.mark.parametrize("which", ["jittered", "cubic"])
def test_ray_integral_exact_filter_drops_no_tet(which):
    """The bounding-box prefilter loses nothing: with and without it the exact
    rational sums are equal (100 rays, half of them starting inside the mesh)."""
    v, t = W.kuhn_cube(3)
    verts = W.jitter_interior(v, t, 3, W.rng_for(2, 43)) if which == "jittered" else W.cubic_map(v)
    rng = np.random.default_rng(102)
    S, T = W.random_rays_through_box(100, rng)
    S[50:] = rng.uniform(-0.9, 0.9, size=(50, 3))     # sources inside the mesh
    mu = rng.uniform(0.0, 1.0, size=t.shape[0])
    nonzero = 0
    for k in range(100):
        a = exact.ray_integral_exact(verts, t, mu, S[k], T[k])
        b = exact.ray_integral_exact(verts, t, mu, S[k], T[k], pad=None)
        assert a == b, (k, a, b)
        nonzero += a > 0
    assert nonzero > 60


# ------------------------------------------------------------ forward_rays_range

def _golden_partial():
    rows = []
    with open(os.path.join(GOLDEN, "single_tet_partial_chords.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def test_forward_rays_range_golden_unit_tet(oracle_lib):
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    rows = _golden_partial()
    assert len(rows) >= 8
    R = np.array(rows)
    got = oracle_lib.forward_rays_range(verts, tets, np.ones(1), R[:, 0:3], R[:, 3:6],
                                        R[:, 6], R[:, 7])
    assert np.all(np.abs(got - R[:, 8]) <= 1e-15 * np.maximum(R[:, 8], 1.0)), (got, R[:, 8])


def test_forward_rays_range_full_and_additive(oracle_lib):
    """[0, inf) is forward_rays; [0, s] + [s, inf) = [0, inf) for any s."""
    verts, tets = W.kuhn_cube(4)
    verts = W.jitter_interior(verts, tets, 4, W.rng_for(2, 44))
    rng = np.random.default_rng(103)
    S, T = W.random_rays_through_box(200, rng)
    S[100:] = rng.uniform(-0.9, 0.9, size=(100, 3))
    mu = rng.uniform(0.0, 1.0, size=tets.shape[0])
    full = oracle_lib.forward_rays(verts, tets, mu, S, T)
    r0 = oracle_lib.forward_rays_range(verts, tets, mu, S, T, 0.0, np.inf)
    assert np.array_equal(full, r0)
    for s in (1.0, rng.uniform(0.2, 1.5, size=200)):
        a = oracle_lib.forward_rays_range(verts, tets, mu, S, T, 0.0, s)
        b = oracle_lib.forward_rays_range(verts, tets, mu, S, T, s, np.inf)
        assert np.all(np.abs(a + b - full) <= 1e-13 * np.maximum(full, 1e-3))
        assert (a > 0).sum() > 50 and (b > 0).sum() > 50
    # a range past the hull or before t = 0 holds nothing
    assert np.all(oracle_lib.forward_rays_range(verts, tets, mu, S, T, 50.0, np.inf) == 0.0)


# ------------------------------------------------- forward_rays_exact_planar

# Kuhn 4^3 arrangement planes n . x = c (n primitive, first non-zero component
# positive) with one ray inside each, all coordinates dyadic so that the ray
# lies in the plane exactly; P is inside the cube so both limits are non-empty.
PLANES = [
    ((1, 0, 0), 0.5, (0.5, -4.0, 0.3125), (0.5, 0.25, -0.125)),
    ((0, 1, 0), 0.0, (-4.0, 0.0, 0.3125), (0.3125, 0.0, -0.25)),
    ((0, 0, 1), -0.5, (4.0, 0.3125, -0.5), (-0.25, -0.125, -0.5)),
    ((1, -1, 0), 0.5, (4.5, 4.0, 0.3125), (0.25, -0.25, -0.125)),
    ((1, 0, -1), 0.0, (4.0, 0.3125, 4.0), (-0.25, 0.125, -0.25)),
    ((0, 1, -1), -0.5, (0.3125, -4.5, -4.0), (0.125, 0.25, 0.75)),
]


@pytest.mark.parametrize("n,c,S,P", PLANES)
def test_forward_rays_exact_planar_closed_form(oracle_lib, n, c, S, P):
    """The symbolic perturbation S + (e, e^2, e^4) puts the line, for t < 1, on
    the side of the plane where the first non-zero component of n grows, and
    beyond P (t > 1) on the other side.  With mu = 1 on the tets of the positive
    side (resp. negative side) the integral is the cube chord over t in [0, 1]
    (resp. [1, inf)); with mu = 1 everywhere it is the whole cube chord."""
    verts, tets = W.kuhn_cube(4)
    S = np.array([S])
    P = np.array([P])
    assert exact.face_planes_containing(verts, tets, S[0], P[0]) == [tuple(n)]
    cen = W.tet_centroids(verts, tets)
    s = cen @ np.array(n, float) - c
    assert np.all(np.abs(s) > 1e-3)        # every Kuhn tet is on one side
    pos = (s > 0).astype(float)
    iv = exact.cube_interval(S[0], P[0])
    assert iv is not None and float(iv[0]) < 1.0 < float(iv[1])
    want_pos = _chord(iv, S[0], P[0], 0.0, 1.0)
    want_neg = _chord(iv, S[0], P[0], 1.0)
    got_pos = oracle_lib.forward_rays_exact_planar(verts, tets, pos, S, P)[0]
    got_neg = oracle_lib.forward_rays_exact_planar(verts, tets, 1.0 - pos, S, P)[0]
    got_all = oracle_lib.forward_rays_exact_planar(verts, tets, np.ones(tets.shape[0]), S, P)[0]
    assert want_pos > 0.5 and want_neg > 0.1
    assert abs(got_pos - want_pos) <= 1e-13 * want_pos, (got_pos, want_pos)
    assert abs(got_neg - want_neg) <= 1e-13 * want_neg, (got_neg, want_neg)
    assert abs(got_all - (want_pos + want_neg)) <= 1e-13 * got_all


def test_forward_rays_exact_planar_rejects_bad_inputs(oracle_lib):
    verts, tets = W.kuhn_cube(4)
    one = np.ones(tets.shape[0])
    with pytest.raises(oracle.PlanarSideError):      # in no face plane
        oracle_lib.forward_rays_exact_planar(verts, tets, one, np.array([[4.0, 0.1, 0.2]]),
                                             np.array([[-4.0, 0.3, 0.1]]))
    # the concrete direction is checked against the symbolic sign: a normal
    # whose leading component is 1e-7 of the next one would get the wrong side
    oracle.check_side_direction([(1, 0, 0), (1, -1, 0), (0, 1, -1), (0, 0, 1)])
    with pytest.raises(oracle.PlanarSideError):
        oracle.check_side_direction([(1, -10 ** 7, 0)])
    with pytest.raises(oracle.PlanarSideError):
        oracle.check_side_direction([(0, 1, -10 ** 7)])


# ------------------------------------------------------------ ray_in_face_plane

def test_ray_in_face_plane_constructed():
    v, t = W.kuhn_cube(4)
    # in-plane rays of every Kuhn plane orientation, and their one-ulp nudges
    for n, c, S, P in PLANES:
        S = np.array(S)
        P = np.array(P)
        assert exact.ray_in_face_plane(v, t, S, P)
        for k in range(3):
            Q = P.copy()
            Q[k] = np.nextafter(Q[k], np.inf)
            assert exact.ray_in_face_plane(v, t, S, Q) == (n[k] == 0 and
                                                           len(exact.face_planes_containing(v, t, S, Q)) > 0)
    # jittered mesh: the line of a face edge lies in that face's plane; generic rays lie in none
    verts = W.jitter_interior(v, t, 4, W.rng_for(2, 45))
    rng = np.random.default_rng(104)
    for i in rng.choice(t.shape[0], size=20, replace=False):
        a, b = verts[t[i, 0]], verts[t[i, 1]]
        assert exact.ray_in_face_plane(verts, t, a, b)
    S, T = W.random_rays_through_box(30, rng)
    assert not any(exact.ray_in_face_plane(verts, t, S[k], T[k]) for k in range(30))
