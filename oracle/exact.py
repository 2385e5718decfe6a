"""Exact rational geometry for pinning -- TEST INFRASTRUCTURE ONLY.

Every FP64 input is converted to a ``fractions.Fraction`` (exactly), so signs
and parameters below are exact.  This module is independent of both the C
oracle (which clips with plane equations in FP64) and the CUDA library.

Contents
--------
side(S, P, p, q)
    The Pluecker side of the line through S, P against the directed edge p->q:
    det[P - S, p - S, q - S].  Its sign says on which side of the edge line the
    ray line passes (Sec. II-C uses four triangle tests per tet; a triangle is
    crossed iff the three edge sides agree in sign).
side_sos(S, P, p, q)
    Sign of ``side`` for the symbolically perturbed line through
    S + (e, e^2, e^4) and P + (e^8, e^16, e^32), e -> 0+.  This is the tie-break
    used where the paper only asks for an unspecified check on zero-length
    intersections (Alg. 2): perturbing the *line*, not the vertices, makes every
    tet see the same perturbed ray, so the walk can neither leak nor loop.
side_sos_bruteforce(S, P, p, q, eps)
    Sign of the exact determinant for that perturbed line at a concrete tiny
    rational eps; pins ``side_sos``.
plucker_interval(V, S, P)
    Exact parameter interval of the line inside a tet, found from the
    barycentric coordinates of the crossing points (edge sides as weights),
    not from plane equations; pins the oracle's Cyrus-Beck clipper.
kuhn_crossings(n, S, P)
    Exact count of positive-length pieces of a ray in the unjittered Kuhn
    split of [-1,1]^n-cells: the split is the arrangement of the planes
    x_i = (2k - n)/n and x_i - x_j = 2k/n.
cube_interval(S, P)
    Exact parameter interval of the half-line in [-1, 1]^3.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from typing import Sequence

Vec = Sequence


def fr3(v) -> tuple:
    return tuple(Fr(float(x)) for x in v)


def sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def det3(r0, r1, r2):
    return dot(r0, cross(r1, r2))


def sign(x) -> int:
    return (x > 0) - (x < 0)


def side(S, P, p, q) -> Fr:
    S, P, p, q = fr3(S), fr3(P), fr3(p), fr3(q)
    return det3(sub(P, S), sub(p, S), sub(q, S))


def _sos_coefficients(S, P, p, q):
    """Coefficients of side(S + s, P + r, p, q) in powers of e, for
    s = (e, e^2, e^4), r = (e^8, e^16, e^32), listed by increasing exponent.

    side is affine in S and in P (it is a 4x4 determinant with rows (S,1),
    (P,1), (p,1), (q,1)), so the expansion has a constant term, terms linear in
    s and in r, and a bilinear term (q - p).(s x r).
      d side / dS = -(p - P) x (q - P)       (exponents 1, 2, 4)
      d side / dP =  (p - S) x (q - S)       (exponents 8, 16, 32)
      (q - p).(s x r): s_i r_j has exponent 2^i + 2^(3+j).
    """
    S, P, p, q = fr3(S), fr3(P), fr3(p), fr3(q)
    d2 = sub(q, p)
    cs = cross(sub(p, P), sub(q, P))
    cs = (-cs[0], -cs[1], -cs[2])
    cr = cross(sub(p, S), sub(q, S))
    terms = {0: det3(sub(P, S), sub(p, S), sub(q, S))}
    for i in range(3):
        terms[1 << i] = cs[i]
        terms[1 << (3 + i)] = cr[i]
    e = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    for i in range(3):
        for j in range(3):
            k = (1 << i) + (1 << (3 + j))
            terms[k] = terms.get(k, 0) + dot(d2, cross(e[i], e[j]))
    return [terms[k] for k in sorted(terms)]


def side_sos(S, P, p, q) -> int:
    for c in _sos_coefficients(S, P, p, q):
        if c != 0:
            return sign(c)
    return 0  # only when p == q


def side_sos_bruteforce(S, P, p, q, eps: Fr = Fr(1, 2 ** 40)) -> int:
    """Exact sign of the determinant for the perturbed line at a concrete eps.

    Equals side_sos when eps is small enough that the lowest non-zero
    coefficient dominates the rest (true for the inputs of the tests, whose
    coefficients are bounded and whose exponents differ by >= 1)."""
    S, P, p, q = fr3(S), fr3(P), fr3(p), fr3(q)
    s = (eps, eps ** 2, eps ** 4)
    r = (eps ** 8, eps ** 16, eps ** 32)
    S2 = tuple(S[i] + s[i] for i in range(3))
    P2 = tuple(P[i] + r[i] for i in range(3))
    return sign(det3(sub(P2, S2), sub(p, S2), sub(q, S2)))


def orient3d(a, b, c, d) -> Fr:
    a, b, c, d = fr3(a), fr3(b), fr3(c), fr3(d)
    return det3(sub(b, a), sub(c, a), sub(d, a))


# Local faces of a positively oriented tet (v0, v1, v2, v3): face f is opposite
# v_f; the triple is ordered so that orient3d(a, b, c, v_f) > 0.
FACE_TRIPLE = {0: (1, 3, 2), 1: (0, 2, 3), 2: (0, 3, 1), 3: (0, 1, 2)}


def plucker_interval(V, S, P):
    """Exact (t_in, t_out) of the line S + t (P - S) inside tet V [4][3], or None.

    A face (a, b, c), ordered so the opposite vertex is on its positive side,
    is crossed inward iff side(a->b), side(b->c), side(c->a) are all > 0 and
    outward iff all < 0 (for rays crossing no edge).  The crossing point is
    X = (w_a a + w_b b + w_c c) / (w_a + w_b + w_c) with w_a = side(b->c),
    w_b = side(c->a), w_c = side(a->b), and t = (X - S).(P - S) / |P - S|^2.
    The interval is NOT clipped to t >= 0 here.
    """
    Vf = [fr3(v) for v in V]
    if orient3d(*Vf) < 0:
        Vf[2], Vf[3] = Vf[3], Vf[2]
    Sf, Pf = fr3(S), fr3(P)
    d = sub(Pf, Sf)
    dd = dot(d, d)
    t_in = t_out = None
    for f, (i, j, k) in FACE_TRIPLE.items():
        a, b, c = Vf[i], Vf[j], Vf[k]
        wc = det3(d, sub(a, Sf), sub(b, Sf))
        wa = det3(d, sub(b, Sf), sub(c, Sf))
        wb = det3(d, sub(c, Sf), sub(a, Sf))
        if (wa > 0 and wb > 0 and wc > 0) or (wa < 0 and wb < 0 and wc < 0):
            W = wa + wb + wc
            X = tuple((wa * a[m] + wb * b[m] + wc * c[m]) / W for m in range(3))
            t = dot(sub(X, Sf), d) / dd
            if wa > 0:
                t_in = t
            else:
                t_out = t
    if t_in is None or t_out is None:
        return None
    return t_in, t_out


def cube_interval(S, P, half: Fr = Fr(1)):
    """Exact parameter interval of the half-line (t >= 0) inside [-half, half]^3."""
    Sf, Pf = fr3(S), fr3(P)
    d = sub(Pf, Sf)
    lo, hi = Fr(0), None
    for i in range(3):
        if d[i] == 0:
            if not (-half <= Sf[i] <= half):
                return None
            continue
        t1 = (-half - Sf[i]) / d[i]
        t2 = (half - Sf[i]) / d[i]
        if t1 > t2:
            t1, t2 = t2, t1
        lo = max(lo, t1)
        hi = t2 if hi is None else min(hi, t2)
    if hi is None or hi <= lo:
        return None
    return lo, hi


def box_interval(S, P, lo_corner, hi_corner):
    """Exact parameter interval of the half-line inside an axis-aligned box."""
    Sf, Pf = fr3(S), fr3(P)
    d = sub(Pf, Sf)
    lo, hi = Fr(0), None
    for i in range(3):
        a, b = Fr(lo_corner[i]), Fr(hi_corner[i])
        if d[i] == 0:
            if not (a <= Sf[i] <= b):
                return None
            continue
        t1 = (a - Sf[i]) / d[i]
        t2 = (b - Sf[i]) / d[i]
        if t1 > t2:
            t1, t2 = t2, t1
        lo = max(lo, t1)
        hi = t2 if hi is None else min(hi, t2)
    if hi is None or hi <= lo:
        return None
    return lo, hi


def kuhn_crossings(n: int, S, P):
    """(#positive-length pieces, in_plane) of the half-line in the Kuhn split of
    [-1,1]^3 into n^3 cells.  in_plane is True when the ray lies inside one of
    the arrangement's planes (then the count is not meaningful)."""
    iv = cube_interval(S, P)
    if iv is None:
        return 0, False
    t0, t1 = iv
    Sf, Pf = fr3(S), fr3(P)
    d = sub(Pf, Sf)
    ts = set()
    for i in range(3):
        if d[i] == 0:
            for k in range(n + 1):
                if Sf[i] == Fr(2 * k - n, n):
                    return 0, True
            continue
        for k in range(n + 1):
            t = (Fr(2 * k - n, n) - Sf[i]) / d[i]
            if t0 < t < t1:
                ts.add(t)
    for i in range(3):
        for j in range(i + 1, 3):
            dd = d[i] - d[j]
            ss = Sf[i] - Sf[j]
            if dd == 0:
                for k in range(-n, n + 1):
                    if ss == Fr(2 * k, n):
                        return 0, True
                continue
            for k in range(-n, n + 1):
                t = (Fr(2 * k, n) - ss) / dd
                if t0 < t < t1:
                    ts.add(t)
    return 1 + len(ts), False


def _int_scale(vals):
    """Exact integers m_k with vals[k] = m_k * 2^E for a common E (all finite doubles)."""
    import math
    parts = []
    for v in vals:
        m, e = math.frexp(v)  # v = m * 2^e, 0.5 <= |m| < 1
        parts.append((int(m * (1 << 53)), e - 53))
    E = min(e for _, e in parts)
    return [m << (e - E) for m, e in parts]


def side_sign_int(S, P, p, q) -> int:
    """Exact sign of det[P - S, p - S, q - S] with Python integers (fast path
    for large test batches; same value as side())."""
    vals = [float(x) for x in (*S, *P, *p, *q)]
    I = _int_scale(vals)
    s, Pp, pp, qq = I[0:3], I[3:6], I[6:9], I[9:12]
    a = [Pp[i] - s[i] for i in range(3)]
    b = [pp[i] - s[i] for i in range(3)]
    c = [qq[i] - s[i] for i in range(3)]
    det = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
           + a[2] * (b[0] * c[1] - b[1] * c[0]))
    return (det > 0) - (det < 0)


class DegenerateRay(ValueError):
    """The ray meets an edge or vertex exactly: crossing faces are not unique."""


def _bbox_candidates(V, S, P, pad, half_line):
    """Indices of tets whose padded bounding box meets the line S + t (P - S)
    (t >= 0 only when half_line).  A coarse float filter: pad widens every box
    so that rounding in the slab test cannot drop a tet the line touches."""
    import numpy as np
    d = P - S
    lo = V.min(axis=1) - pad
    hi = V.max(axis=1) + pad
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        inv = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), np.inf)
        t1 = (lo - S) * inv
        t2 = (hi - S) * inv
    tmin = np.where(d != 0, np.minimum(t1, t2), np.where((S >= lo) & (S <= hi), -np.inf, np.inf))
    tmax = np.where(d != 0, np.maximum(t1, t2), np.where((S >= lo) & (S <= hi), np.inf, -np.inf))
    keep = tmin.max(axis=1) <= tmax.min(axis=1) * (1 + 1e-12) + 1e-12
    if half_line:
        keep &= tmax.min(axis=1) >= -1e-12
    return np.nonzero(keep)[0]


def ray_integral_exact(verts, tets, mu, S, P, pad=1e-9):
    """Exact sum_i a_ij mu_i for one ray (Eq. 2) with a_ij from exact integer
    arithmetic: each tet's crossing points come from barycentric weights given
    by exact side products (as in plucker_interval), clipped to t >= 0.  Only
    tets whose bounding box meets the ray (padded by ``pad``) are examined;
    ``pad=None`` examines every tet (used to check that the filter drops none).
    Raises DegenerateRay if a crossing is not unique (a zero side product on a
    crossed face).  Returns a float (the exact rational sum, rounded)."""
    import math
    import numpy as np
    S = np.asarray(S, float)
    P = np.asarray(P, float)
    d = P - S
    V = np.asarray(verts, float)[np.asarray(tets)]          # [nt, 4, 3]
    if pad is None:
        cand = np.arange(V.shape[0])
    else:
        cand = _bbox_candidates(V, S, P, pad, half_line=True)
    # common integer scaling of every coordinate involved
    vals = list(S) + list(P) + list(V[cand].reshape(-1))
    I = _int_scale([float(x) for x in vals])
    Si, Pi = I[0:3], I[3:6]
    di = [Pi[k] - Si[k] for k in range(3)]
    dd = sum(x * x for x in di)

    def det(a, b, c):
        return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
                + a[2] * (b[0] * c[1] - b[1] * c[0]))

    total = Fr(0)
    for q, i in enumerate(cand):
        base = 6 + 12 * q
        v = [I[base + 3 * k: base + 3 * k + 3] for k in range(4)]
        rel = [[v[k][m] - Si[m] for m in range(3)] for k in range(4)]
        o = det([v[1][m] - v[0][m] for m in range(3)], [v[2][m] - v[0][m] for m in range(3)],
                [v[3][m] - v[0][m] for m in range(3)])
        if o < 0:
            rel[2], rel[3] = rel[3], rel[2]
        t_in = t_out = None
        for f, (ia, ib, ic) in FACE_TRIPLE.items():
            a, b, c = rel[ia], rel[ib], rel[ic]
            wc = det(di, a, b)
            wa = det(di, b, c)
            wb = det(di, c, a)
            pos = wa > 0 and wb > 0 and wc > 0
            neg = wa < 0 and wb < 0 and wc < 0
            if not (pos or neg):
                if (wa == 0 or wb == 0 or wc == 0) and \
                        ((wa >= 0 and wb >= 0 and wc >= 0) or (wa <= 0 and wb <= 0 and wc <= 0)):
                    if wa or wb or wc:
                        raise DegenerateRay(int(i))
                continue
            W = wa + wb + wc
            num = sum((wa * a[m] + wb * b[m] + wc * c[m]) * di[m] for m in range(3))
            t = Fr(num, W * dd)
            if pos:
                t_in = t
            else:
                t_out = t
        if t_in is None or t_out is None:
            continue
        t0 = max(t_in, Fr(0))
        if t_out > t0:
            total += (t_out - t0) * Fr(float(mu[i]))
    return float(total) * math.sqrt(float(d @ d))


def _int_det(a, b, c):
    return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
            + a[2] * (b[0] * c[1] - b[1] * c[0]))


def face_planes_containing(verts, tets, S, P, pad=1e-9, return_kappa=False):
    """Normals of the face planes that contain the line S->P exactly.

    Exact integer orientation tests over the tets whose (padded) bounding box
    meets the line.  Each normal is the integer triple (b - a) x (c - a) of the
    face's vertices on a common integer grid, divided by the gcd of its
    components, with a positive first non-zero component, so its components
    (their signs and ratios) are exact; faces in one plane give one normal.
    With ``return_kappa`` a dict {normal: E} is returned instead: per component
    k, E_k is the largest |e1_i e2_j| + |e1_j e2_i| ((i, j) the other two
    components; e1, e2 two edges of a face of the plane from any of its
    vertices, on the same scale as the normal), so that an FP64 cross product
    of FP64 edge vectors differs from the normal by at most ~4 u E_k in
    component k -- and by nothing where both products are exactly zero."""
    import math
    import numpy as np
    S = np.asarray(S, float)
    P = np.asarray(P, float)
    V = np.asarray(verts, float)[np.asarray(tets)]
    cand = _bbox_candidates(V, S, P, pad, half_line=False)
    vals = list(S) + list(P) + list(V[cand].reshape(-1))
    I = _int_scale([float(x) for x in vals])
    Si, Pi = I[0:3], I[3:6]
    out = {}
    for q in range(cand.size):
        base = 6 + 12 * q
        v = [I[base + 3 * k: base + 3 * k + 3] for k in range(4)]
        for f in range(4):
            a, b, c = [v[k] for k in range(4) if k != f]
            e1 = [b[m] - a[m] for m in range(3)]
            e2 = [c[m] - a[m] for m in range(3)]
            if _int_det(e1, e2, [Si[m] - a[m] for m in range(3)]) == 0 and \
                    _int_det(e1, e2, [Pi[m] - a[m] for m in range(3)]) == 0:
                n = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                     e1[0] * e2[1] - e1[1] * e2[0]]
                E = [0, 0, 0]
                for p0, p1, p2 in ((a, b, c), (b, c, a), (c, a, b)):
                    f1 = [p1[m] - p0[m] for m in range(3)]
                    f2 = [p2[m] - p0[m] for m in range(3)]
                    for k_, (i, j) in enumerate(((1, 2), (2, 0), (0, 1))):
                        E[k_] = max(E[k_], abs(f1[i] * f2[j]) + abs(f1[j] * f2[i]))
                g = math.gcd(math.gcd(abs(n[0]), abs(n[1])), abs(n[2]))
                n = [x // g for x in n]
                lead = next(x for x in n if x != 0)
                if lead < 0:
                    n = [-x for x in n]
                key = tuple(n)
                prev = out.get(key, (0.0, 0.0, 0.0))
                out[key] = tuple(max(prev[m], E[m] / g) for m in range(3))
    if return_kappa:
        return out
    return sorted(out)


def ray_in_face_plane(verts, tets, S, P, pad=1e-9):
    """True if the line S->P lies exactly in the plane of a face of a tet whose
    bounding box it meets (exact integer orientation tests)."""
    return len(face_planes_containing(verts, tets, S, P, pad)) > 0


def sos_side_sign(n) -> int:
    """Sign of n . (e, e^2, e^4) as e -> 0+: the sign of the first non-zero
    component of n.  This is the side of a plane with normal n that the
    symbolically perturbed source S + (e, e^2, e^4) lies on."""
    for x in n:
        if x != 0:
            return 1 if x > 0 else -1
    return 0
