"""Full-size parity (GPU): the bench workload and the robustness workload.

* Jittered Kuhn 96^3, 512 x 512 x 360 rays, in the launch configuration the
  bench times (filtered FP32, default options): sampled rays against the
  oracle's brute-force clip, sampled tets' backprojections against the
  oracle's sums over all 94M rays, and the adjoint identity.
* Cubic-mapped Kuhn 64^3 (spacing ratio ~3e3) with 256^2 x 180 detector rays
  and 1M adversarial rays aimed exactly at vertices, edge midpoints and face
  points: no walk fails in either precision, and sampled rays match the oracle
  (exact references for rays inside or 1e-16 off a face plane).  The measured
  errors are printed (they are reported per configuration in the design notes).

Tolerances as in test_gpu_parity (tau * sum a|mu| + 16 u R max|mu|).
"""
import numpy as np
import pytest

import oracle
import workloads as W

from test_gpu_parity import TOL, floor_abs, planar_reference

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


def _rel_report(name, got, want, scale):
    rel = np.abs(got - want) / np.maximum(scale, 1e-300)
    print(f"{name}: max rel {rel.max():.3e}  median rel {np.median(rel):.3e}  n={rel.size}")


def test_bench_workload_sampled(tp):
    import torch
    w = W.config2()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    mu = torch.tensor(w.mu, dtype=torch.float32, device="cuda")
    mesh.stats_reset()
    proj = tp.forward(mesh, geo, mu)
    back = tp.backward(mesh, geo, proj)
    st = mesh.stats()
    assert st["error"] == 0
    rng = np.random.default_rng(51)
    idx = np.sort(rng.choice(geo.nrays, 96, replace=False))
    S, P = oracle.cone_rays(w.geom, idx)
    want = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom, idx)
    scale = oracle.forward_cone(w.verts, w.tets, np.abs(w.mu), w.geom, idx)
    _, _, _, _, _, planar = oracle.trace_rays(w.verts, w.tets, S, P, max_visits=2)
    assert not planar.any()
    got = proj.reshape(-1)[torch.tensor(idx, device="cuda")].double().cpu().numpy()
    _rel_report("C2 forward f32", got, want, scale)
    assert np.all(np.abs(got - want) <= TOL["f32"] * scale + floor_abs("f32", w.verts, w.mu))
    # backprojection of the projection, at 6 tets crossed by many rays
    y = proj.double().cpu().numpy().reshape(-1)
    cen = W.tet_centroids(w.verts, w.tets)
    near = np.nonzero(np.linalg.norm(cen, axis=1) < 0.5)[0]
    tets = rng.choice(near, 6, replace=False)
    wantb = oracle.backward_cone_subset(w.verts, w.tets, y, w.geom, tets)
    gotb = back[torch.tensor(tets, device="cuda")].double().cpu().numpy()
    _rel_report("C2 backward f32 (y >= 0)", gotb, wantb, wantb)
    assert np.all(np.abs(gotb - wantb) <= TOL["f32"] * wantb)
    # adjoint identity at full size
    g = torch.Generator("cuda").manual_seed(3)
    x = torch.rand(mesh.nt, device="cuda", generator=g) - 0.5
    yy = torch.rand(geo.shape, device="cuda", generator=g) - 0.5
    lhs = float((tp.forward(mesh, geo, x).double() * yy.double()).sum())
    rhs = float((x.double() * tp.backward(mesh, geo, yy).double()).sum())
    mag = float((tp.forward(mesh, geo, x.abs()).double() * yy.double().abs()).sum())
    assert abs(lhs - rhs) <= TOL["f32"] * mag


@pytest.fixture(scope="module")
def c3():
    return W.config3()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_robustness_workload(tp, c3, prec):
    import torch
    w = c3
    dt = torch.float32 if prec == "f32" else torch.float64
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    mu = torch.tensor(w.mu, dtype=dt, device="cuda")
    mesh.stats_reset()
    proj = tp.forward(mesh, geo, mu)
    AS, AT = w.extra["adv_src"], w.extra["adv_target"]
    adv = tp.forward_rays(mesh, torch.tensor(AS, device="cuda"), torch.tensor(AT, device="cuda"), mu)
    st = mesh.stats()
    print(prec, st)
    assert st["error"] == 0 and st["error_count"] == 0
    assert st["sos"] > 0
    rng = np.random.default_rng(61)
    fl = floor_abs(prec, w.verts, w.mu)
    # detector rays
    idx = np.sort(rng.choice(geo.nrays, 48, replace=False))
    S, P = oracle.cone_rays(w.geom, idx)
    want = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom, idx)
    _, _, _, _, _, planar = oracle.trace_rays(w.verts, w.tets, S, P, max_visits=2)
    ref = planar_reference(w.verts, w.tets, w.mu, S, P, want, planar)
    got = proj.reshape(-1)[torch.tensor(idx, device="cuda")].double().cpu().numpy()
    _rel_report(f"C3 detector {prec}", got, ref["want"], want)
    assert np.all(np.abs(got - ref["want"]) <= TOL[prec] * want + fl)
    # adversarial rays: a sample of each kind
    kind = w.extra["adv_kind"]
    sel = np.concatenate([rng.choice(np.nonzero(kind == k)[0], 24, replace=False) for k in range(3)])
    want = oracle.forward_rays(w.verts, w.tets, w.mu, AS[sel], AT[sel])
    _, _, _, _, _, planar = oracle.trace_rays(w.verts, w.tets, AS[sel], AT[sel], max_visits=2)
    ref = planar_reference(w.verts, w.tets, w.mu, AS[sel], AT[sel], want, planar)
    got = adv[torch.tensor(sel, device="cuda")].double().cpu().numpy()
    ok = np.ones(sel.size, bool)
    ok[ref["skipped"]] = False
    _rel_report(f"C3 adversarial {prec}", got[ok], ref["want"][ok], want[ok])
    assert np.all(np.abs(got - ref["want"])[ok] <= TOL[prec] * want[ok] + fl)


@pytest.mark.parametrize("k", [8, 18, 12])
def test_batched_workload_problem_sampled(tp, k):
    """Full-size problems of the batched workload (config 5) through the batched
    launch: #8 (34^3 cells, 1022^2 x 310 rays) and #18 (27^3, 811^2 x 451) put
    ~10^5 segments into each tet, #12 is the largest mesh (118^3, 9.9M tets).
    4 channels; sampled rays against the oracle's clipping, sampled central
    tets' backprojections of the projection against the oracle's sums."""
    import torch
    n, N, na = W.config5_specs()[k]
    w = W.config5_problem(k, n, N, na, channels=4)
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    b = tp.Batch([mesh], [geo], channels=4, tiles=[(16, 8, tp.ORDER_MORTON, tp.SCATTER_ATOMIC)])
    b.mu[0].copy_(torch.tensor(w.mu, dtype=torch.float32))
    b.forward()
    b.y[0].copy_(b.proj[0])
    b.backward()
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    rng = np.random.default_rng(300 + k)
    idx = np.sort(rng.choice(geo.nrays, 48, replace=False))
    want = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom, idx)
    scale = oracle.forward_cone(w.verts, w.tets, np.abs(w.mu), w.geom, idx)
    S, P = oracle.cone_rays(w.geom, idx)
    planar = oracle.trace_rays(w.verts, w.tets, S, P, max_visits=2)[5]
    got = b.proj[0].reshape(-1, 4)[torch.tensor(idx, device="cuda")].double().cpu().numpy()
    ok = ~planar
    _rel_report(f"C5#{k} forward f32", got[ok], want[ok], scale[ok])
    assert np.all((np.abs(got - want) <= TOL["f32"] * scale + floor_abs("f32", w.verts, w.mu))[ok])
    cen = W.tet_centroids(w.verts, w.tets)
    near = np.nonzero(np.linalg.norm(cen, axis=1) < 0.3)[0]
    tets = rng.choice(near, 3, replace=False)
    y = b.y[0].double().cpu().numpy().reshape(-1, 4)
    wantb = oracle.backward_cone_subset(w.verts, w.tets, y, w.geom, tets)
    gotb = b.mu_out[0][torch.tensor(tets, device="cuda")].double().cpu().numpy()
    _rel_report(f"C5#{k} backward f32", gotb, wantb, wantb)
    assert np.all(np.abs(gotb - wantb) <= TOL["f32"] * wantb)
    b.close()


def test_fp64_accumulator_many_segments_per_tet(tp):
    """Problem #18 of the batched workload (27^3 cells, 811^2 x 451 rays, ~10^5
    segments per tet): FP32 atomic sums (TETPROJ_FLAG_ACC32) come within 1e-5 of
    the oracle only just; the FP64 accumulator (the default at C = 1) keeps ~1e-7."""
    import torch
    k = 18
    n, N, na = W.config5_specs()[k]
    w = W.config5_problem(k, n, N, na, channels=1)
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    mu = torch.tensor(w.mu[:, 0], dtype=torch.float32, device="cuda")
    y = tp.forward(mesh, geo, mu)
    b32 = tp.backward(mesh, geo, y, options=tp.make_options(flags=tp.FLAG_ACC32))
    b64 = tp.backward(mesh, geo, y)  # the default for C = 1
    rng = np.random.default_rng(318)
    cen = W.tet_centroids(w.verts, w.tets)
    tets = rng.choice(np.nonzero(np.linalg.norm(cen, axis=1) < 0.3)[0], 4, replace=False)
    wantb = oracle.backward_cone_subset(w.verts, w.tets, y.double().cpu().numpy().reshape(-1),
                                        w.geom, tets)
    idx = torch.tensor(tets, device="cuda")
    g32 = b32[idx].double().cpu().numpy()
    g64 = b64[idx].double().cpu().numpy()
    _rel_report("C5#18 backward f32 accumulator", g32, wantb, wantb)
    _rel_report("C5#18 backward f64 accumulator", g64, wantb, wantb)
    assert np.all(np.abs(g64 - wantb) <= 1e-6 * wantb)
