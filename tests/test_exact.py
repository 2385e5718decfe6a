"""Pins for the exact rational predicates (no GPU)."""
from fractions import Fraction as Fr

import numpy as np

from oracle import exact


def test_side_matches_float_det_when_well_conditioned():
    rng = np.random.default_rng(1)
    for _ in range(300):
        S, P, p, q = rng.normal(size=(4, 3))
        want = np.linalg.det(np.array([P - S, p - S, q - S]))
        got = exact.side(S, P, p, q)
        if abs(want) > 1e-6:
            assert exact.sign(got) == np.sign(want)
            assert abs(float(got) - want) <= 1e-12 * (1 + abs(want))


def test_side_is_pluecker_product():
    """side = d.(p x q) + (q - p).(S x P): the permuted inner product of the
    ray line (d, S x P) and the edge line (q - p, p x q)."""
    rng = np.random.default_rng(2)
    for _ in range(100):
        S, P, p, q = [exact.fr3(v) for v in rng.normal(size=(4, 3))]
        d = exact.sub(P, S)
        want = exact.dot(d, exact.cross(p, q)) + exact.dot(exact.sub(q, p), exact.cross(S, P))
        assert exact.side(S, P, p, q) == want


def test_orient3d_unit():
    assert exact.orient3d([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]) == 1
    assert exact.orient3d([0, 0, 0], [0, 1, 0], [1, 0, 0], [0, 0, 1]) == -1


def _degenerate_cases(rng, n):
    """Exactly degenerate (S, P, p, q): vertex-through, collinear, coplanar."""
    out = []
    grid = lambda: rng.integers(-4, 5, size=3).astype(float) / 4.0
    for _ in range(n):
        kind = rng.integers(0, 5)
        p, q = grid(), grid()
        while np.all(p == q):
            q = grid()
        S = grid() * 4
        if kind == 0:      # ray aimed exactly at p
            P = p.copy()
        elif kind == 1:    # ray through p, beyond
            P = p + (p - S)
        elif kind == 2:    # ray coplanar with the edge (crosses its line)
            P = S + (p - S) + 0.5 * (q - p) * rng.integers(1, 4)
        elif kind == 3:    # ray along the edge line
            S = p - 2.0 * (q - p)
            P = q.copy()
        else:              # parallel to the edge
            P = S + (q - p)
        out.append((S, P, p, q))
    return out


def test_sos_matches_bruteforce_perturbation():
    rng = np.random.default_rng(3)
    cases = _degenerate_cases(rng, 300)
    zeros = 0
    for S, P, p, q in cases:
        if exact.side(S, P, p, q) == 0:
            zeros += 1
        s = exact.side_sos(S, P, p, q)
        assert s in (-1, 1)
        assert s == exact.side_sos_bruteforce(S, P, p, q, Fr(1, 2 ** 30))
    assert zeros > 200


def test_sos_antisymmetric_and_consistent():
    rng = np.random.default_rng(4)
    for S, P, p, q in _degenerate_cases(rng, 200):
        assert exact.side_sos(S, P, p, q) == -exact.side_sos(S, P, q, p)
        v = exact.side(S, P, p, q)
        if v != 0:
            assert exact.side_sos(S, P, p, q) == exact.sign(v)


def test_sos_walk_consistency_on_vertex_ray():
    """A ray aimed exactly at a vertex: the perturbed signs around one tet still
    select exactly one exit face (one sign change in the cyclic order)."""
    n = np.array([0.0, 0.0, 1.0])
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    S = np.array([0.25, 0.25, -3.0])
    for P in (n, b, (a + b) * 0.5):
        s = [exact.side_sos(S, P, n, k) for k in (a, b, c)]
        changes = sum(1 for i in range(3) if s[i] > 0 and s[(i + 1) % 3] < 0)
        assert changes == 1, s


def test_kuhn_crossings_small():
    # ray along x through cell interiors of the n=2 split: cube [-1,1],
    # planes x=-1,0,1 and x-y=k, x-z=k: crosses x=0, x-y=0 (y=0.3), x-z=0 (z=0.6)...
    S = np.array([-3.0, 0.3, 0.6])
    P = np.array([3.0, 0.3, 0.6])
    cnt, inplane = exact.kuhn_crossings(2, S, P)
    # breakpoints inside (-1,1): x=0, x=0.3 (x-y=0), x=0.6 (x-z=0), x=-0.7 (x-y=-1),
    # x=-0.4 (x-z=-1): 5 distinct -> 6 pieces
    assert (cnt, inplane) == (6, False)
