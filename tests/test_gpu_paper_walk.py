"""The paper's own walk (Alg. 1-2: Moller-Trumbore + growing eps) as a
comparison mode, GPU.

* Parity: the CUDA comparison mode and the C reference of the same steps
  (oracle/mt.c) take the same decisions in FP32 and in FP64 -- identical
  per-ray status (done / halted / step limit) and equal sums -- on a jittered
  mesh with detector rays and on a cubic-mapped (high aspect ratio) mesh with
  rays aimed exactly at vertices, edge midpoints and face points.
* On generic rays the FP64 walk agrees with the plain definition (oracle.c).
* The floating-point experiment of Sec. III-C on the robustness workload
  (cubic-mapped Kuhn 64^3, 256^2 x 180 rays + 1M adversarial rays): rays
  that halt or loop in FP32 and FP64 Alg. 1-2, against the exact-predicate
  filtered walk (no failures).  Counts are printed and recorded in the design
  notes.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

MAX_STEPS = 2000


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


def _opts(tp, prec):
    return tp.make_options(precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64,
                           tile=(8, 8), max_steps=MAX_STEPS)


def _mu(x, prec):
    """mu as the precision sees it (FP32 values kept exactly in FP64)."""
    return x.astype(np.float32).astype(np.float64) if prec == "f32" else x


def _compare(got, got_st, want, want_st, prec, label):
    same_status = np.array_equal(got_st, want_st)
    ok = want_st == 0
    bit_equal = np.mean(got[ok] == want[ok]) if ok.any() else 1.0
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    print(f"{label} {prec}: status equal {same_status}, halted {int((want_st == 1).sum())}, "
          f"loops {int((want_st == 2).sum())}, bit-equal sums {bit_equal:.4f}, max rel {rel.max():.2e}")
    assert same_status
    tol = 1e-5 if prec == "f32" else 1e-13
    assert np.all(rel <= tol)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_paper_walk_matches_reference_detector_rays(tp, prec):
    import torch
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(6, 1))
    mu = _mu(W.rng_for(6, 2).uniform(0, 1, tets.shape[0]), prec)
    geom = W.ConeBeam(4.0, 8.0, 24, 20, 0.25, 0.25, W.uniform_angles(16) + 0.05)
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry.from_cone(geom)
    dt = torch.float32 if prec == "f32" else torch.float64
    got, st = tp.forward_mt(mesh, geo, torch.tensor(mu, dtype=dt, device="cuda"),
                            options=_opts(tp, prec))
    S, P = oracle.cone_rays(geom)
    # the library caps the step limit at nt + 1 (no walk visits more tets)
    want, want_st = oracle.mt_forward_rays(verts, tets, mu, S, P, prec,
                                           min(MAX_STEPS, tets.shape[0] + 1))
    _compare(got.double().cpu().numpy().reshape(-1), st.cpu().numpy().reshape(-1), want, want_st,
             prec, "detector rays")
    if prec == "f64":
        exact = oracle.forward_cone(verts, tets, mu, geom)
        scale = oracle.forward_cone(verts, tets, np.abs(mu), geom)
        assert np.all(np.abs(want - exact) <= 1e-12 * scale + 1e-15)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_paper_walk_matches_reference_adversarial(tp, prec):
    import torch
    n = 12
    verts, tets = W.kuhn_cube(n)
    verts = W.cubic_map(verts)
    mu = _mu(W.rng_for(6, 3).uniform(0, 1, tets.shape[0]), prec)
    AS, AT, kind = W.adversarial_rays(verts, tets, n, 3000, W.rng_for(6, 4))
    mesh = tp.Mesh(verts, tets)
    dt = torch.float32 if prec == "f32" else torch.float64
    got, st = tp.forward_rays_mt(mesh, torch.tensor(AS, device="cuda"),
                                 torch.tensor(AT, device="cuda"),
                                 torch.tensor(mu, dtype=dt, device="cuda"),
                                 options=_opts(tp, prec))
    want, want_st = oracle.mt_forward_rays(verts, tets, mu, AS, AT, prec,
                                           min(MAX_STEPS, tets.shape[0] + 1))
    _compare(got.double().cpu().numpy(), st.cpu().numpy(), want, want_st, prec, "adversarial rays")


def test_floating_point_experiment_robustness_workload(tp):
    """Sec. III-C: single-precision Alg. 1-2 loses rays (halts / loops) on a mesh
    with large aspect ratios; the exact-predicate walk loses none."""
    import torch
    w = W.config3()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    AS = torch.tensor(w.extra["adv_src"], device="cuda")
    AT = torch.tensor(w.extra["adv_target"], device="cuda")
    rows = {}
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        mu = torch.tensor(w.mu, dtype=dt, device="cuda")
        o = tp.make_options(precision=tp.FILTERED if prec == "f32" else tp.PLAIN_FP64,
                            tile=(8, 8))
        _, st_det = tp.forward_mt(mesh, geo, mu, options=o)
        _, st_adv = tp.forward_rays_mt(mesh, AS, AT, mu, options=o)
        rows[prec] = [int((s == k).sum()) for s in (st_det, st_adv) for k in (1, 2)]
    mesh.stats_reset()
    mu32 = torch.tensor(w.mu, dtype=torch.float32, device="cuda")
    proj = tp.forward(mesh, geo, mu32)
    adv = tp.forward_rays(mesh, AS, AT, mu32)
    st = mesh.stats()
    print(f"robustness workload: {geo.nrays} detector rays, {AS.shape[0]} adversarial rays")
    for prec in ("f32", "f64"):
        r = rows[prec]
        print(f"  Alg. 1-2 {prec}: detector halted {r[0]} loops {r[1]}; "
              f"adversarial halted {r[2]} loops {r[3]}")
    print(f"  exact-predicate filtered walk: errors {st['error_count']}, "
          f"NaN outputs {int(torch.isnan(proj).sum()) + int(torch.isnan(adv).sum())}")
    assert st["error_count"] == 0
    assert sum(rows["f32"]) > 0            # the paper's FP32 failure reproduces
    assert sum(rows["f32"]) > sum(rows["f64"])
