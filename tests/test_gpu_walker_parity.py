"""Parity on 10^5 sampled rays per configuration (GPU) against the oracle
walker (oracle.Walker: the brute-force clipper's a_ij, found by walking the
oracle's own adjacency; pinned in test_oracle_walker).

* Config 2 (the bench workload) and config 4, both precisions: the forward
  projection at 10^5 seeded rays, and the backprojection of a y that is
  non-zero on those rays only, compared at every tet they cross.
* Config 5, all 24 problems through one batched launch (C = 4, filtered
  FP32): 10^5 rays per problem, forward and backprojection as above; and
  problems #9 and #5 on the plain FP64 path.

Rays the walker finds inside a face plane (status 2: the closed-tet measure
counts both sides there, the method follows one) are left out of the forward
checks and get y = 0 in the backprojections; their references are the exact
ones of test_gpu_parity / test_gpu_fullsize.

Tolerances, from the arithmetic.  Rounding moves a crossing point along the
ray by about u (L + R) kappa / sin(alpha): L its distance from the source, R
the mesh radius, alpha the angle between ray and face plane, kappa the
crossed face's shape factor (sum of squared edges / 2|n|: sqrt 3 for an
equilateral face, ~1 / sin of the smallest angle for a sliver, by which the
rounding of the face normal's cross product turns it).  The crossing is a
ratio of two quantities each computed to a few u of magnitudes proportional
to sin(alpha) -- in the oracle's clipper and in both GPU paths.  A ray's
integral moves by the crossing's shift times the jump of mu there; a tet's
backprojection by the shifts of its two crossings times y.  The walker sums
these per ray (K_j = sum |mu jump| (L + R) kappa / sin) and per tet
(K_i = sum_j |y_j| ((L + R) kappa / sin)_in + ((L + R) kappa / sin)_out).
Bounds:
  per ray  |b_gpu - b_ref| <= max(tau sum_i a_ij |mu_i|, 32 e K_j)
  per tet  |x_gpu - x_ref| <= max(tau sum_j a_ij |y_j|, 32 e K_i)
with e = 2^-53 on the FP64 path, and on the FP32 path e K = 2^-24 K(1 / sin
capped at 64) + 2^-53 K (crossings with sin below 1/64 are placed again in
FP64).  32 covers both sides' errors (each ~13 u (L + R) kappa / sin: the
cross product, the two dot products and the division).  tau is 1e-5 (FP32)
or 1e-12 (FP64) relative.  Each check prints how many rays or tets only the
conditioning term admits.  A ray through an edge or vertex touches tets with
a_ij = 0 that a computed walk may visit with a chord of its rounding's size:
the walker's rows for such rays list those tets, so their conditioning is in
K_i.  Tets that no sampled ray crosses or touches must stay below
64 * 32 u R max|y|.
"""
import numpy as np
import pytest

import oracle
import workloads as W

from test_gpu_parity import TOL, UNIT

pytestmark = pytest.mark.gpu

NSAMPLE = 100_000


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


def _dt(prec):
    import torch
    return torch.float32 if prec == "f32" else torch.float64


def sample(nrays, seed, n=NSAMPLE):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nrays, min(n, nrays), replace=False)), rng


def cond_term(prec, K):
    """32 e K (module doc): K [..., 2] = (1 / sin capped at 64, uncapped)."""
    K = np.asarray(K, np.float64)
    if prec == "f32":
        return 32.0 * (UNIT["f32"] * K[..., 0] + UNIT["f64"] * K[..., 1])
    return 32.0 * UNIT["f64"] * K[..., 1]


def check_cond(name, got, want, scale, K, prec, skip=None):
    """|got - want| <= max(tau scale, 32 e K) elementwise (rows: rays or tets,
    columns: channels); prints the errors and how many rows only the
    conditioning term admits.  Rows in `skip` (a boolean mask) are left out."""
    got = np.asarray(got, np.float64).reshape(K.shape[0], -1)
    want = np.asarray(want, np.float64).reshape(K.shape[0], -1)
    scale = np.asarray(scale, np.float64).reshape(K.shape[0], -1)
    keep = np.ones(K.shape[0], bool) if skip is None else ~skip
    err = np.abs(got - want)[keep]
    rel = TOL[prec] * scale[keep]
    cond = cond_term(prec, K)[keep]
    bound = np.maximum(rel, cond)
    only = np.any(err > rel, axis=1)
    r = err / np.maximum(scale[keep], 1e-300)
    worst = float((err / np.maximum(cond, 1e-300))[only].max()) if only.any() else 0.0
    print(f"{name}: n={err.shape[0]} max rel {r.max():.3e} median rel {np.median(r):.3e} "
          f"max abs {err.max():.3e}; admitted only by the conditioning term: {int(only.sum())} "
          f"(largest error / term {worst:.3f})")
    bad = np.nonzero(np.any(err > bound, axis=1))[0]
    assert bad.size == 0, (name, bad[:5], err[bad[:5]], bound[bad[:5]])
    return int(only.sum())


def touched(cnt, Kb):
    """Tets a sampled ray crosses, or only touches (walker rows not walked
    list those with a_ij = 0 and their crossings' conditioning)."""
    return (cnt > 0) | (np.asarray(Kb)[..., 1].reshape(cnt.size, -1).max(axis=1) > 0)


def check_uncrossed(name, got, cnt, prec, R, ymax):
    """Tets no sampled ray crosses or touches (cnt: 0 for those, 1 for the
    others): |x_gpu| <= 64 * 32 u R max|y|."""
    got = np.asarray(got, np.float64).reshape(cnt.size, -1)
    stray = float(np.abs(got[cnt == 0]).max()) if (cnt == 0).any() else 0.0
    q = 32.0 * UNIT[prec] * R * ymax
    print(f"{name}: largest value at a tet no sampled ray crosses {stray:.3e}")
    assert stray <= 64 * q, (name, stray, 64 * q)


def planar_free_y(wk, geom, idx, rng, C):
    """y for the sampled rays: U[0.5, 1.5] (FP32-representable), but 0 on
    rays that lie inside a face plane (walker status 2), whose split between
    the tets on either side of the plane is not unique."""
    _, st = wk.forward_cone(np.zeros((wk.nt, C)), geom, idx)
    y = rng.uniform(0.5, 1.5, size=(idx.size, C)).astype(np.float32).astype(np.float64)
    y[st == 2] = 0.0
    return y


def scatter_sample(geo_shape, C, idx, vals, dt):
    """A full-size y (geo_shape, or geo_shape + (C,)) on the device, zero but
    at the sampled rays."""
    import torch
    y = torch.zeros(int(np.prod(geo_shape)), C, dtype=dt, device="cuda")
    y[torch.tensor(idx, device="cuda")] = torch.tensor(vals.reshape(-1, C), dtype=dt, device="cuda")
    return y.view(*geo_shape, C) if C > 1 else y.view(*geo_shape)


class Single:
    """One mesh, its walker and a 10^5-ray sample with the oracle's rows:
    forward of (mu, |mu|) and backprojection of y >= 0 on the sample."""

    def __init__(self, tp, w, seed):
        self.w = w
        self.mesh = tp.Mesh(w.verts, w.tets)
        self.geo = tp.Geometry.from_cone(w.geom)
        self.idx, rng = sample(self.geo.nrays, seed)
        mu = np.asarray(w.mu, np.float64)
        self.C = 1 if mu.ndim == 1 else mu.shape[1]
        wk = oracle.Walker(w.verts, w.tets)
        # FP32-representable y in [0.5, 1.5], 0 on rays inside a face plane
        self.yv = planar_free_y(wk, w.geom, self.idx, rng, self.C)
        m2 = np.concatenate([mu.reshape(-1, self.C), np.abs(mu).reshape(-1, self.C)], axis=1)
        y2 = np.concatenate([self.yv, self.yv], axis=1)
        fwd, bwd, self.status = wk.rows_cone(m2, y2, w.geom, self.idx)
        self.want, self.scale = fwd[:, :self.C], fwd[:, self.C:]
        self.wantb = bwd[:, :self.C]
        self.cnt = wk.last_count
        self.kf, self.kb = wk.last_kf[:, :self.C], wk.last_kb[:, :self.C]
        self.planar = self.status == 2
        print(f"{w.name}: walker status counts {np.bincount(self.status, minlength=3)}")

    def run(self, tp, prec, options=None, backward=None):
        import torch
        dt = _dt(prec)
        mu = torch.tensor(np.asarray(self.w.mu), dtype=dt, device="cuda")
        self.mesh.stats_reset()
        proj = tp.forward(self.mesh, self.geo, mu, options=options)
        y = scatter_sample(self.geo.shape, self.C, self.idx, self.yv, dt)
        back = (backward or tp.backward)(self.mesh, self.geo, y, options=options)
        torch.cuda.synchronize()
        assert self.mesh.stats()["error"] == 0
        got = proj.reshape(-1, self.C)[torch.tensor(self.idx, device="cuda")].double().cpu().numpy()
        return got, back.double().cpu().numpy()

    def check(self, tp, prec, options=None, backward=None, label=""):
        got, back = self.run(tp, prec, options, backward)
        w = self.w
        R = float(np.abs(w.verts).max())
        check_cond(f"{w.name}{label} forward {prec} (10^5 rays, {int(self.planar.sum())} in-plane left out)",
                   got, self.want, self.scale, self.kf, prec, skip=self.planar)
        hit = touched(self.cnt, self.kb)
        check_cond(f"{w.name}{label} backward {prec} ({int(hit.sum())} tets crossed)", back[hit],
                   self.wantb[hit], self.wantb[hit], self.kb[hit], prec)
        check_uncrossed(f"{w.name}{label} backward {prec}", back, hit.astype(np.int64), prec, R,
                        float(self.yv.max()))


@pytest.fixture(scope="module")
def c2(tp):
    return Single(tp, W.config2(), 61)


@pytest.fixture(scope="module")
def c4(tp):
    return Single(tp, W.config4(), 62)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_config2_walker_sampled(tp, c2, prec):
    c2.check(tp, prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_config4_walker_sampled(tp, c4, prec):
    c4.check(tp, prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_config3_detector_rays_walker_sampled(tp, prec):
    """Config 3's detector rays (cubic-mapped Kuhn 64^3, spacing ratio ~3e3:
    sliver tets near the centre), 10^5 of them, both precisions."""
    Single(tp, W.config3(n_adversarial=0), 63).check(tp, prec)


@pytest.mark.parametrize("scatter", ["warp", "sort"])
def test_config2_scatter_variants_walker_sampled(tp, c2, scatter):
    """The two other backprojection scatters on the bench workload (FP32):
    warp-aggregated reductions into the FP64 accumulator, and the
    deterministic segment sort-and-reduce."""
    sc = tp.SCATTER_WARP if scatter == "warp" else tp.SCATTER_SORT
    c2.check(tp, "f32", tp.make_options(scatter=sc), label=f" ({scatter} scatter)")


def test_config4_backward_noalloc_walker_sampled(tp, c4):
    """The allocation-free backprojection (fixed device scratch) on the
    config-4 mesh (1.57M tets: within its 32 MB accumulator at C = 1)."""
    c4.check(tp, "f32", backward=lambda m, g, y, options=None: tp.backward_noalloc(m, g, y),
             label=" (noalloc backprojection)")


@pytest.mark.parametrize("k", [12, 18])
def test_config5_single_calls_fp32_walker_sampled(tp, k):
    """Config-5 problems through single calls (filtered FP32, 4 channels):
    #12, the largest mesh (118^3), and #18 (~10^5 segments per tet, two-level
    accumulation)."""
    n, N, na = W.config5_specs()[k]
    s = Single(tp, W.config5_problem(k, n, N, na, channels=4), 720 + k)
    s.check(tp, "f32", tp.make_options(channels=4))


@pytest.mark.parametrize("k", [9, 5])
def test_config5_plain_fp64_walker_sampled(tp, k):
    n, N, na = W.config5_specs()[k]
    s = Single(tp, W.config5_problem(k, n, N, na, channels=4), 700 + k)
    s.check(tp, "f64", tp.make_options(precision=tp.PLAIN_FP64, channels=4))


def test_config5_all_problems_batched_walker_sampled(tp):
    """All 24 problems in one batched launch (the bench's batched workload at
    full size, default tiles), 10^5 rays per problem."""
    import torch
    specs = W.config5_specs()
    ws = [W.config5_problem(k, n, N, na, channels=4) for k, (n, N, na) in enumerate(specs)]
    meshes = [tp.Mesh(w.verts, w.tets) for w in ws]
    geos = [tp.Geometry.from_cone(w.geom) for w in ws]
    b = tp.Batch(meshes, geos, channels=4)
    samples = []
    for k, w in enumerate(ws):
        idx, rng = sample(geos[k].nrays, 800 + k)
        yv = planar_free_y(oracle.Walker(w.verts, w.tets), w.geom, idx, rng, 4)
        samples.append((idx, yv))
        b.mu[k].copy_(torch.tensor(w.mu, dtype=torch.float32))
        b.y[k].copy_(scatter_sample(geos[k].shape, 4, idx, yv, torch.float32).reshape(b.y[k].shape))
    b.forward()
    b.backward()
    torch.cuda.synchronize()
    for k, w in enumerate(ws):
        assert meshes[k].stats()["error"] == 0, k
        idx, yv = samples[k]
        wk = oracle.Walker(w.verts, w.tets)
        mu = np.asarray(w.mu, np.float64)  # U[0, 1]: sum a|mu| is the value itself
        fwd, bwd, st = wk.rows_cone(mu, yv, w.geom, idx)
        cnt = wk.last_count
        planar = st == 2
        got = b.proj[k].reshape(-1, 4)[torch.tensor(idx, device="cuda")].double().cpu().numpy()
        check_cond(f"C5#{k} batched forward f32, 4 channels ({int(planar.sum())} in-plane left out)",
                   got, fwd, fwd, wk.last_kf, "f32", skip=planar)
        back = b.mu_out[k].double().cpu().numpy()
        hit = touched(cnt, wk.last_kb)
        check_cond(f"C5#{k} batched backward f32 ({int(hit.sum())} tets crossed)", back[hit],
                   bwd[hit], bwd[hit], wk.last_kb[hit], "f32")
        check_uncrossed(f"C5#{k} batched backward f32", back, hit.astype(np.int64), "f32",
                        float(np.abs(w.verts).max()), float(yv.max()))
        del wk
    b.close()


def _visit_workload(name):
    if name == "C2":
        return W.config2()
    if name == "C3":
        return W.config3(n_adversarial=0)
    if name == "C4":
        return W.config4()
    k = int(name[3:])  # "C5#k"
    n, N, na = W.config5_specs()[k]
    return W.config5_problem(k, n, N, na, channels=4)


@pytest.mark.parametrize("name", ["C2", "C3", "C4", "C5#12", "C5#0"])
def test_visit_sequences_full_size(tp, name):
    """Identical tet-visit sequences on 10^4 sampled rays of each full-size
    configuration (the walker's non-degenerate rays: no two candidate
    crossings within 1e-9), in both precisions, with each visit's chord within
    32 e K of the oracle's (K the visit's two crossings' (L + R) / sin)."""
    import torch
    w = _visit_workload(name)
    mesh = tp.Mesh(w.verts, w.tets)
    idx, _ = sample(w.geom.nrays, 900 + len(name), n=10_000)
    S, P = oracle.cone_rays(w.geom, idx)
    wk = oracle.Walker(w.verts, w.tets)
    mv = 1024
    tet, ln, cnt, st = wk.trace_rays(S, P, max_visits=mv)
    cond = wk.last_cond
    sel = np.nonzero((st == 0) & (cnt > 0) & (cnt <= mv))[0]
    assert sel.size > 0.5 * np.count_nonzero(cnt)
    src = torch.tensor(S[sel], device="cuda")
    dst = torch.tensor(P[sel], device="cuda")
    for prec in ("f32", "f64"):
        gt, gl, gc = tp.trace_rays(mesh, src, dst, max_visits=mv,
                                   precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64)
        torch.cuda.synchronize()
        gt, gl, gc = gt.cpu().numpy(), gl.cpu().numpy(), gc.cpu().numpy()
        assert np.array_equal(gc, cnt[sel]), (name, prec)
        worst = 0.0
        nvis = 0
        for r, k in enumerate(sel):
            n = cnt[k]
            assert np.array_equal(gt[r, :n], tet[k, :n]), (name, prec, k)
            err = np.abs(gl[r, :n] - ln[k, :n])
            bound = cond_term(prec, cond[k, :n])
            assert np.all(err <= np.maximum(bound, 1e-300)), (name, prec, k, (err / bound).max())
            worst = max(worst, float((err / bound).max()))
            nvis += n
        print(f"{name} visit sequences {prec}: {sel.size} rays, {nvis} visits identical; "
              f"largest chord error / 32 e K {worst:.3f}")
    assert mesh.stats()["error"] == 0


def test_config3_adversarial_rays_walker_sampled(tp):
    """10^4 of config 3's adversarial rays (aimed exactly at vertices, edge
    midpoints and face points of the cubic-mapped mesh; 3,334 / 3,333 / 3,333
    per kind), both precisions, against the oracle (their walks meet ties, so
    most rows come from the clipper through the walker's fallback); rays
    inside a face plane are left out (exact references in test_gpu_fullsize)."""
    import torch
    w = W.config3()
    mesh = tp.Mesh(w.verts, w.tets)
    AS, AT, kind = w.extra["adv_src"], w.extra["adv_target"], w.extra["adv_kind"]
    rng = np.random.default_rng(950)
    sel = np.concatenate([rng.choice(np.nonzero(kind == k)[0], 3334 - (k > 0), replace=False)
                          for k in range(3)])
    S, P = AS[sel], AT[sel]
    wk = oracle.Walker(w.verts, w.tets)
    mu = np.asarray(w.mu)  # U[0, 1]: sum a|mu| is the value itself
    want, _, st = wk.rows_rays(mu, None, S, P)
    want = want[:, 0]
    K = wk.last_kf
    planar = st == 2
    print(f"C3 adversarial: walker status counts {np.bincount(st, minlength=3)}")
    src = torch.tensor(S, device="cuda")
    dst = torch.tensor(P, device="cuda")
    for prec in ("f32", "f64"):
        o = tp.make_options(precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64)
        got = tp.forward_rays(mesh, src, dst, torch.tensor(mu, dtype=_dt(prec), device="cuda"),
                              options=o)
        torch.cuda.synchronize()
        check_cond(f"C3 adversarial forward {prec} ({int(planar.sum())} in-plane left out)",
                   got.double().cpu().numpy(), want, want, K, prec, skip=planar)
    # the explicit-ray backprojection of y >= 0 on these rays (0 on in-plane ones)
    yv = rng.uniform(0.5, 1.5, size=sel.size).astype(np.float32).astype(np.float64)
    yv[planar] = 0.0
    _, wantb, _ = wk.rows_rays(None, yv, S, P)
    wantb = wantb[:, 0]
    cnt, Kb = wk.last_count, wk.last_kb
    hit = touched(cnt, Kb)
    for prec in ("f32", "f64"):
        o = tp.make_options(precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64)
        back = tp.backward_rays(mesh, src, dst, torch.tensor(yv, dtype=_dt(prec), device="cuda"),
                                options=o)
        torch.cuda.synchronize()
        back = back.double().cpu().numpy()
        check_cond(f"C3 adversarial backward {prec} ({int(hit.sum())} tets crossed)", back[hit],
                   wantb[hit], wantb[hit], Kb[hit], prec)
        check_uncrossed(f"C3 adversarial backward {prec}", back, hit.astype(np.int64), prec,
                        float(np.abs(w.verts).max()), 1.5)
    assert mesh.stats()["error"] == 0
