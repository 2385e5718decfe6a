"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances.  Per ray: |b_gpu - b_ref| <= max(tau * sum_i a_ij |mu_i|,
32 u R max|mu|), with tau = 1e-12 (plain FP64) or 1e-5 (filtered FP32), u the
unit roundoff of the path (2^-53 or 2^-24) and R the largest |coordinate| of
the mesh.  The second term is the coordinate quantum: crossing points are
placed in the path's coordinates, each a few u R off (rounding of the vertices,
the weights and the point itself; grazing crossings are placed again in FP64),
so rays that only clip a corner (sum a|mu| below 32 u R max|mu| / tau, i.e.
chords shorter than ~0.2 R in FP32) are held to it instead; every longer ray
is held to tau.  How many rays pass only through the floor is counted and
bounded.  Per tet: tau * sum_j a_ij |y_j|.

References.  b_ref is the oracle's brute-force clip, except for rays the
oracle flags as (nearly) inside a face plane, where FP64 clipping cannot tell
the two sides apart:
* a ray EXACTLY in a face plane (exact integer test) has no unique integral;
  the method follows the symbolically perturbed line, whose limit is the
  one-sided integral on the side of the source perturbation up to t = 1 and on
  the other side beyond (oracle.forward_rays_exact_planar);
* a ray only NEAR a face plane (e.g. 1e-16 off it because cos(pi/2) != 0) has
  a unique integral, computed in exact integer arithmetic
  (oracle.exact.ray_integral_exact).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import exact

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


def floor_abs(prec, verts, mu):
    return 32.0 * UNIT[prec] * float(np.abs(verts).max()) * float(np.abs(mu).max())


@pytest.fixture(scope="module")
def tp():
    import torch
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    import paper_1908_06909_gb300 as tp
    return tp


def _dt(prec):
    import torch
    return torch.float64 if prec == "f64" else torch.float32


def _side_dir(seed, n):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(n, 3))
    return w / np.linalg.norm(w, axis=1, keepdims=True)


class C1Data:
    def __init__(self, tp):
        self.w = W.config1()
        w = self.w
        self.mesh = tp.Mesh(w.verts, w.tets)
        self.geo = tp.Geometry.from_cone(w.geom)
        self.S, self.P = oracle.cone_rays(w.geom)
        tt, lo, hi, cnt, margin, planar = oracle.trace_rays(w.verts, w.tets, self.S, self.P,
                                                            max_visits=128)
        self.tr = (tt, lo, hi, cnt, margin, planar)
        self.planar = planar
        self.b = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom)
        self.scale = oracle.forward_cone(w.verts, w.tets, np.abs(w.mu), w.geom)
        self.planar_idx = np.nonzero(planar)[0]
        self.ref = planar_reference(w.verts, w.tets, w.mu, self.S, self.P, self.b, planar)
        assert self.ref["n_exact_plane"] > 0 and self.ref["n_near_plane"] > 0


@pytest.fixture(scope="module")
def c1(tp):
    return C1Data(tp)


def planar_reference(verts, tets, mu, S, P, b, planar):
    """Reference values for oracle-flagged planar rays (see module doc)."""
    want = np.array(b, dtype=np.float64, copy=True)
    n_exact = n_near = 0
    skipped = []
    for k in np.nonzero(planar)[0]:
        if exact.ray_in_face_plane(verts, tets, S[k], P[k]):
            want[k] = oracle.forward_rays_exact_planar(verts, tets, mu, S[k:k + 1], P[k:k + 1])[0]
            n_exact += 1
        else:
            try:
                want[k] = exact.ray_integral_exact(verts, tets, mu, S[k], P[k])
                n_near += 1
            except exact.DegenerateRay:
                skipped.append(k)
    return {"want": want, "n_exact_plane": n_exact, "n_near_plane": n_near, "skipped": skipped}


def check_rays(name, got, want, scale, tol, floor, skip=(), max_floor_frac=0.01):
    """Per-ray parity with the short-chord floor (module doc); prints the
    errors and how many rays only the floor admits, and bounds that count."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    want = np.asarray(want, dtype=np.float64).reshape(-1)
    scale = np.asarray(scale, dtype=np.float64).reshape(-1)
    ok = np.ones(got.size, bool)
    ok[list(skip)] = False
    err = np.abs(got[ok] - want[ok])
    rel = tol * scale[ok]
    bound = np.maximum(rel, floor)
    worst = np.argmax(err - bound)
    n_floor = int(np.sum(err > rel))
    r = err / np.maximum(scale[ok], 1e-300)
    print(f"{name}: n={err.size} max rel {r.max():.3e} median rel {np.median(r):.3e} "
          f"max abs {err.max():.3e}; admitted only by the floor: {n_floor}")
    assert np.all(err <= bound), (f"{name}: max rel err {r.max():.3e}, "
                                  f"worst abs {err[worst]:.3e} vs bound {bound[worst]:.3e} "
                                  f"(ray {np.nonzero(ok)[0][worst]})")
    assert n_floor <= max(3, max_floor_frac * err.size), (name, n_floor)
    return n_floor



@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_forward_c1(tp, c1, prec):
    import torch
    mu = torch.tensor(c1.w.mu, dtype=_dt(prec), device="cuda")
    c1.mesh.stats_reset()
    proj = tp.forward(c1.mesh, c1.geo, mu)
    torch.cuda.synchronize()
    assert proj.shape == (32, 64, 64)
    assert c1.planar_idx.size > 0  # C1 contains rays lying in Kuhn face planes
    check_rays(f"C1 forward {prec}", proj.double().cpu().numpy(), c1.ref["want"], c1.scale,
               TOL[prec], floor_abs(prec, c1.w.verts, c1.w.mu), c1.ref["skipped"])
    assert len(c1.ref["skipped"]) < 8
    st = c1.mesh.stats()
    assert st["error"] == 0 and st["rays"] == 131072
    assert st["hits"] == int((c1.scale > 0).sum())


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_backward_c1(tp, c1, prec):
    import torch
    rng = np.random.default_rng(31)
    y = rng.uniform(0, 1, size=c1.geo.nrays)
    y[c1.planar_idx] = 0.0  # per-tet values of in-plane rays are ambiguous
    want = oracle.backward_cone(c1.w.verts, c1.w.tets, y, c1.w.geom)
    scale = want  # y >= 0
    yt = torch.tensor(y.reshape(c1.geo.shape), dtype=_dt(prec), device="cuda")
    got = tp.backward(c1.mesh, c1.geo, yt).double().cpu().numpy()
    err = np.abs(got - want)
    assert np.all(err <= TOL[prec] * np.maximum(scale, 1e-300) + 1e-300), err.max()
    assert (want > 0).sum() > 2000


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_closed_form_chord(tp, c1, prec):
    import torch
    one = torch.ones(c1.mesh.nt, dtype=_dt(prec), device="cuda")
    got = tp.forward(c1.mesh, c1.geo, one).double().cpu().numpy().reshape(-1)
    rng = np.random.default_rng(4)
    sel = rng.choice(got.size, 3000, replace=False)
    want = np.zeros(sel.size)
    for r, k in enumerate(sel):
        iv = exact.cube_interval(c1.S[k], c1.P[k])
        d = c1.P[k] - c1.S[k]
        want[r] = 0.0 if iv is None else float(iv[1] - iv[0]) * float(np.sqrt(d @ d))
    check_rays(f"C1 closed-form chord {prec}", got[sel], want, want, TOL[prec],
               floor_abs(prec, c1.w.verts, [1.0]))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_visit_sequences(tp, c1, prec):
    """Identical tet-visit sequences on non-degenerate rays."""
    import torch
    tt, lo, hi, cnt, margin, planar = c1.tr
    rng = np.random.default_rng(5)
    cand = np.nonzero((margin > 1e-9) & (~planar) & (cnt > 0))[0]
    sel = rng.choice(cand, 3000, replace=False)
    src = torch.tensor(c1.S[sel], device="cuda")
    dst = torch.tensor(c1.P[sel], device="cuda")
    gt, gl, gc = tp.trace_rays(c1.mesh, src, dst, max_visits=128,
                               precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64)
    gt, gl, gc = gt.cpu().numpy(), gl.cpu().numpy(), gc.cpu().numpy()
    dlen = np.linalg.norm(c1.P[sel] - c1.S[sel], axis=1)
    for r, k in enumerate(sel):
        n = cnt[k]
        assert gc[r] == n, (k, gc[r], n)
        assert np.array_equal(gt[r, :n], tt[k, :n])
        want = (hi[k, :n] - lo[k, :n]) * dlen[r]
        assert np.all(np.abs(gl[r, :n] - want) <= (1e-12 if prec == "f64" else 2e-6) * 4)


class MappedData:
    """A 16^3-cell Kuhn mesh, jittered (config 2/4 style) or cubic-mapped
    (config 3 style), with the oracle's rows of A for 64 x 64 x 4 cone rays."""

    def __init__(self, tp, kind):
        n = 16
        v, t = W.kuhn_cube(n)
        self.verts = W.jitter_interior(v, t, n, W.rng_for(1, 161)) if kind == "jittered" \
            else W.cubic_map(v)
        self.tets = t
        self.geom = W.ConeBeam(4.0, 8.0, 64, 64, 0.1, 0.1, W.uniform_angles(4))
        self.S, self.P = oracle.cone_rays(self.geom)
        self.tr = oracle.trace_rays(self.verts, t, self.S, self.P, max_visits=192)
        self.mesh = tp.Mesh(self.verts, t)


@pytest.fixture(scope="module", params=["jittered", "cubic"])
def mapped(tp, request):
    return MappedData(tp, request.param)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_visit_sequences_mapped_meshes(tp, mapped, prec):
    """Identical tet-visit sequences on non-degenerate rays through a jittered
    and a cubic-mapped mesh (tets of uneven size and shape), with each visit's
    chord against the oracle's clipped interval."""
    import torch
    tt, lo, hi, cnt, margin, planar = mapped.tr
    assert cnt.max() < 192
    rng = np.random.default_rng(6)
    cand = np.nonzero((margin > 1e-9) & (~planar) & (cnt > 0))[0]
    sel = rng.choice(cand, 3000, replace=False)
    src = torch.tensor(mapped.S[sel], device="cuda")
    dst = torch.tensor(mapped.P[sel], device="cuda")
    gt, gl, gc = tp.trace_rays(mapped.mesh, src, dst, max_visits=192,
                               precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64)
    gt, gl, gc = gt.cpu().numpy(), gl.cpu().numpy(), gc.cpu().numpy()
    dlen = np.linalg.norm(mapped.P[sel] - mapped.S[sel], axis=1)
    worst = 0.0
    for r, k in enumerate(sel):
        n = cnt[k]
        assert gc[r] == n, (k, gc[r], n)
        assert np.array_equal(gt[r, :n], tt[k, :n]), k
        want = (hi[k, :n] - lo[k, :n]) * dlen[r]
        err = np.abs(gl[r, :n] - want)
        worst = max(worst, float(err.max()))
        assert np.all(err <= (1e-12 if prec == "f64" else 2e-6) * 4), (k, err.max())
    print(f"visit sequences {prec}: {sel.size} rays identical, worst chord error {worst:.2e}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_identity(tp, c1, prec):
    import torch
    g = torch.Generator("cuda").manual_seed(7)
    x = torch.rand(c1.mesh.nt, dtype=_dt(prec), device="cuda", generator=g) - 0.5
    y = torch.rand(c1.geo.shape, dtype=_dt(prec), device="cuda", generator=g) - 0.5
    Ax = tp.forward(c1.mesh, c1.geo, x)
    Aty = tp.backward(c1.mesh, c1.geo, y)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * Aty.double()).sum())
    mag = float((tp.forward(c1.mesh, c1.geo, x.abs()).double() * y.double().abs()).sum())
    assert abs(lhs - rhs) <= TOL[prec] * mag


def test_geometry_rays_bit_exact(tp, c1):
    import torch
    src, dst = c1.geo.rays()
    assert np.array_equal(src.cpu().numpy(), c1.S)
    assert np.array_equal(dst.cpu().numpy(), c1.P)
    idx = torch.tensor([0, 5, 131071, 4096], device="cuda")
    s2, d2 = c1.geo.rays(idx)
    assert np.array_equal(d2.cpu().numpy(), c1.P[[0, 5, 131071, 4096]])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_channels_and_rays_api(tp, c1, prec):
    import torch
    rng = np.random.default_rng(8)
    mu4 = rng.uniform(size=(c1.mesh.nt, 4))
    m4 = torch.tensor(mu4, dtype=_dt(prec), device="cuda")
    p4 = tp.forward(c1.mesh, c1.geo, m4)
    for c in range(4):
        p1 = tp.forward(c1.mesh, c1.geo, m4[:, c].contiguous())
        assert torch.allclose(p4[..., c], p1, rtol=TOL[prec], atol=1e-30)
    y4 = torch.tensor(rng.uniform(size=c1.geo.shape + (4,)), dtype=_dt(prec), device="cuda")
    b4 = tp.backward(c1.mesh, c1.geo, y4)
    for c in (0, 3):
        b1 = tp.backward(c1.mesh, c1.geo, y4[..., c].contiguous())
        assert torch.allclose(b4[:, c], b1, rtol=10 * TOL[prec], atol=1e-12)
    # explicit-ray API on the same rays equals the cone-beam call
    src, dst = c1.geo.rays()
    mu = m4[:, 0].contiguous()
    pr = tp.forward_rays(c1.mesh, src, dst, mu)
    pc = tp.forward(c1.mesh, c1.geo, mu).reshape(-1)
    assert torch.allclose(pr, pc, rtol=TOL[prec], atol=1e-30)
    yr = torch.rand(src.shape[0], dtype=_dt(prec), device="cuda")
    br = tp.backward_rays(c1.mesh, src, dst, yr)
    bc = tp.backward(c1.mesh, c1.geo, yr.reshape(c1.geo.shape))
    assert torch.allclose(br, bc, rtol=10 * TOL[prec], atol=1e-12)


def test_side_device_matches_host(tp):
    import torch
    rng = np.random.default_rng(9)
    n = 30000
    p = rng.uniform(-1, 1, size=(n, 3))
    q = p + rng.normal(size=(n, 3)) * 10.0 ** rng.uniform(-5, -1, size=(n, 1))
    X = p + rng.uniform(-0.5, 1.5, size=(n, 1)) * (q - p)
    S = rng.uniform(-4, 4, size=(n, 3))
    P = S + 2 * (X - S) + 10.0 ** rng.uniform(-16, -2, size=(n, 1)) * rng.normal(size=(n, 3))
    # exact zeros too: rays aimed at p
    P[:3000] = p[:3000]
    hs, hst = tp.side_signs_host(S, P, p, q)
    T = lambda a: torch.tensor(a, device="cuda")
    ds, dst = tp.side_signs_device(T(S), T(P), T(p), T(q))
    assert np.array_equal(ds.cpu().numpy(), hs)
    assert np.array_equal(dst.cpu().numpy(), hst)
    assert (hst == 3).sum() >= 3000


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adversarial_rays_small(tp, prec):
    """Rays aimed exactly at vertices, edge midpoints and face points of a
    cubic-mapped Kuhn 8^3 mesh: values equal the oracle (or lie between the
    one-sided limits for rays inside a face plane); no walk fails."""
    import torch
    verts, tets = W.kuhn_cube(8)
    verts = W.cubic_map(verts)
    rng = W.rng_for(2, 9)
    mu = rng.uniform(size=tets.shape[0])
    S, T, kind = W.adversarial_rays(verts, tets, 8, 3000, rng)
    mesh = tp.Mesh(verts, tets)
    _, _, _, _, margin, planar = oracle.trace_rays(verts, tets, S, T, max_visits=4)
    want0 = oracle.forward_rays(verts, tets, mu, S, T)
    scale = want0
    ref = planar_reference(verts, tets, mu, S, T, want0, planar)
    assert ref["n_exact_plane"] > 20
    mesh.stats_reset()
    got = tp.forward_rays(mesh, torch.tensor(S, device="cuda"), torch.tensor(T, device="cuda"),
                          torch.tensor(mu, dtype=_dt(prec), device="cuda"))
    st = mesh.stats()
    assert st["error"] == 0 and st["error_count"] == 0
    assert st["sos"] > 0  # exact zeros were met and resolved symbolically
    check_rays(f"adversarial small {prec}", got.double().cpu().numpy(), ref["want"], scale,
               TOL[prec], floor_abs(prec, verts, mu), ref["skipped"])
    assert len(ref["skipped"]) < 10
    assert (margin < 1e-12).sum() > 1000  # the set really is degenerate


def test_errors_reported(tp, c1):
    import torch
    mu = torch.ones(c1.mesh.nt, dtype=torch.float32, device="cuda")
    o = tp.make_options(max_steps=2)
    c1.mesh.stats_reset()
    proj = tp.forward(c1.mesh, c1.geo, mu, options=o)
    st = c1.mesh.stats()
    assert st["error"] == tp._lib.ERR_RAY_LIMIT and st["error_count"] > 0
    assert torch.isnan(proj).any()
    c1.mesh.stats_reset()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sources_inside_mesh(tp, c1, prec):
    """Half-line semantics (Eq. 1 with t >= 0): sources inside the mesh, and
    rays pointing away from it, integrate only what lies ahead."""
    import torch
    rng = np.random.default_rng(12)
    n = 400
    S = rng.uniform(-0.9, 0.9, size=(n, 3))
    P = S + rng.normal(size=(n, 3))
    S[:50] = rng.uniform(-3, 3, size=(50, 3)) + np.array([6.0, 0, 0])   # mesh behind the source
    P[:50] = S[:50] + np.array([1.0, 0.1, 0.2])
    mu = c1.w.mu
    want = oracle.forward_rays(c1.w.verts, c1.w.tets, mu, S, P)
    c1.mesh.stats_reset()
    got = tp.forward_rays(c1.mesh, torch.tensor(S, device="cuda"), torch.tensor(P, device="cuda"),
                          torch.tensor(mu, dtype=_dt(prec), device="cuda"))
    st = c1.mesh.stats()
    assert st["error"] == 0
    _, _, _, _, _, planar = oracle.trace_rays(c1.w.verts, c1.w.tets, S, P, max_visits=2)
    assert not planar.any()
    check_rays(f"sources inside {prec}", got.double().cpu().numpy(), want, want, TOL[prec],
               floor_abs(prec, c1.w.verts, mu))
    assert np.all(want[:50] == 0) and (want[50:] > 0).all()


def test_empty_and_single_tet(tp):
    import torch
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    T = np.array([[0, 2, 1, 3]])
    mesh = tp.Mesh(V, T)
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    mu = torch.tensor([2.0], dtype=torch.float64, device="cuda")
    assert tp.forward_rays(mesh, e, e, mu).numel() == 0
    out = tp.backward_rays(mesh, e, e, torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert out.shape == (1,) and float(out[0]) == 0.0
    rows = []
    for line in open(__file__.replace("test_gpu_parity.py", "golden/single_tet_chords.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(x) for x in line.split()])
    rows = np.array(rows)
    ok = rows[:, 0] + rows[:, 1] + rows[:, 2] > 1.0 + 1e-9  # sources outside the tet
    ok |= (rows[:, 0:3] < 0).any(axis=1)
    rows = rows[ok]
    src = torch.tensor(rows[:, 0:3], device="cuda")
    dst = torch.tensor(rows[:, 3:6], device="cuda")
    for dt, tol in ((torch.float64, 1e-14), (torch.float32, 1e-6)):
        got = tp.forward_rays(mesh, src, dst, mu.to(dt)).double().cpu().numpy()
        assert np.allclose(got, 2.0 * rows[:, 6], rtol=tol, atol=tol)


@pytest.mark.parametrize("C", [1, 4])
def test_backward_fp64_accumulator_c1(tp, c1, C):
    """Backprojection accumulators: FP64 (TETPROJ_FLAG_ACC64, default at C = 1)
    and FP32 (TETPROJ_FLAG_ACC32, default at C = 4) meet the same oracle bound;
    invalid combinations are rejected."""
    import torch
    w = c1.w
    rng = np.random.default_rng(31 + C)
    y = rng.uniform(-1, 1, size=(c1.geo.nrays, C))
    y[c1.planar] = 0.0
    y = y.astype(np.float32).astype(np.float64)
    yt = torch.tensor(y.reshape(c1.geo.shape + ((C,) if C > 1 else ())), dtype=torch.float32,
                      device="cuda")
    o = tp.make_options(channels=C, flags=tp.FLAG_ACC64)
    got = tp.backward(c1.mesh, c1.geo, yt, options=o).double().cpu().numpy()
    want = oracle.backward_cone(w.verts, w.tets, y if C > 1 else y[:, 0], w.geom)
    scale = oracle.backward_cone(w.verts, w.tets, np.abs(y) if C > 1 else np.abs(y[:, 0]), w.geom)
    assert np.all(np.abs(got - want) <= TOL["f32"] * scale + 1e-30)
    o32 = tp.make_options(channels=C, flags=tp.FLAG_ACC32)
    got32 = tp.backward(c1.mesh, c1.geo, yt, options=o32).double().cpu().numpy()
    assert np.all(np.abs(got32 - want) <= TOL["f32"] * scale + 1e-30)
    # warp-aggregated scatter into the FP64 accumulator (one reduction per tet per warp)
    ow = tp.make_options(channels=C, flags=tp.FLAG_ACC64, scatter=tp.SCATTER_WARP)
    gotw = tp.backward(c1.mesh, c1.geo, yt, options=ow).double().cpu().numpy()
    assert np.all(np.abs(gotw - want) <= TOL["f32"] * scale + 1e-30)
    bad = [dict(flags=tp.FLAG_ACC64, scatter=tp.SCATTER_SORT),   # sort sums runs itself
           dict(flags=tp.FLAG_ACC32, scatter=tp.SCATTER_SORT),
           dict(flags=tp.FLAG_ACC64 | tp.FLAG_ACC32)]
    for kw in bad:
        with pytest.raises(tp.TetprojError):
            tp.backward(c1.mesh, c1.geo, yt, options=tp.make_options(channels=C, **kw))


def test_single_calls_graph_capture_after_reserve(tp):
    """A forward projection and a backprojection of a two-chunk scan (> 2^24
    rays) captured in one CUDA graph on a mesh that only had
    tetproj_mesh_reserve: nothing is allocated under capture (the chunks run
    without the overlap stream), and the replay equals eager calls."""
    import torch
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(4, 900))
    mu_np = W.rng_for(4, 901).uniform(0, 1, tets.shape[0])
    mesh = tp.Mesh(verts, tets)
    mesh.reserve(tp.FILTERED, 1)
    g = W.ConeBeam(4.0, 8.0, 512, 512, 6.4 / 512, 6.4 / 512, W.uniform_angles(68))
    assert g.nrays > 2 ** 24
    geo = tp.Geometry.from_cone(g)
    mu = torch.tensor(mu_np, dtype=torch.float32, device="cuda")
    proj = torch.empty(geo.shape, dtype=torch.float32, device="cuda")
    back = torch.empty(mesh.nt, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        tp.forward(mesh, geo, mu, out=proj)
        tp.backward(mesh, geo, proj, out=back)
    graph.replay()
    torch.cuda.synchronize()
    ref_p = tp.forward(mesh, geo, mu)
    ref_b = tp.backward(mesh, geo, ref_p)
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    assert torch.equal(proj, ref_p)  # per-ray sums: deterministic
    assert torch.allclose(back, ref_b, rtol=1e-6, atol=0)  # FP64 accumulators, any order
    mesh.close()
