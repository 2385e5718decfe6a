"""Sort-and-reduce backprojection (TETPROJ_SCATTER_SORT), GPU.

The deterministic scatter: segments written at positions fixed by the rays'
segment counts, stably radix-sorted by tet, each tet's run summed in order.
Checked: against the oracle (Eq. 3) and the atomic scatter on config 1 (C = 1
and 4), bit-identical results over repeated calls, several chunks (more rays
than one deferral-queue chunk), the full-size bench workload (sampled tets vs
the oracle, repeatability), statistics that count only the real walk, and the
calls that reject it.
"""
import numpy as np
import pytest

import oracle
import workloads as W

from test_gpu_parity import TOL, C1Data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


@pytest.fixture(scope="module")
def c1(tp):
    return C1Data(tp)


def _opts(tp, scatter, C=1, tile=(8, 8), order=None):
    return tp.make_options(precision=tp.FILTERED, channels=C, tile=tile,
                           order=tp.ORDER_MORTON if order is None else order, scatter=scatter)


@pytest.mark.parametrize("C", [1, 4])
def test_sort_matches_oracle_and_atomic_c1(tp, c1, C):
    import torch
    w = c1.w
    rng = np.random.default_rng(91 + C)
    y = rng.uniform(-1, 1, size=(c1.geo.nrays, C))
    y[c1.planar] = 0.0  # rays in face planes: their split between sides is a convention
    y = y.astype(np.float32).astype(np.float64)
    yt = torch.tensor(y.reshape(c1.geo.shape + ((C,) if C > 1 else ())), dtype=torch.float32,
                      device="cuda")
    c1.mesh.stats_reset()
    got = tp.backward(c1.mesh, c1.geo, yt, options=_opts(tp, tp.SCATTER_SORT, C)).double()
    st = c1.mesh.stats()
    assert st["error"] == 0
    assert st["rays"] == c1.geo.nrays  # the plan's counting walk is not counted
    want = oracle.backward_cone(w.verts, w.tets, y if C > 1 else y[:, 0], w.geom)
    scale = oracle.backward_cone(w.verts, w.tets, np.abs(y) if C > 1 else np.abs(y[:, 0]), w.geom)
    g = got.cpu().numpy()
    assert np.all(np.abs(g - want) <= TOL["f32"] * scale + 1e-30)
    atomic = tp.backward(c1.mesh, c1.geo, yt, options=_opts(tp, tp.SCATTER_ATOMIC, C)).double()
    assert np.all(np.abs(g - atomic.cpu().numpy()) <= TOL["f32"] * scale + 1e-30)


def test_sort_is_bit_reproducible_and_plan_reused(tp, c1):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(7)
    y = torch.rand(c1.geo.shape, device="cuda", generator=gen) - 0.5
    o = _opts(tp, tp.SCATTER_SORT, 1, tile=(16, 4), order=tp.ORDER_ROW)
    a = tp.backward(c1.mesh, c1.geo, y, options=o)
    bytes_after_first = c1.mesh.info()["device_bytes"]
    b = tp.backward(c1.mesh, c1.geo, y, options=o)
    c = tp.backward(c1.mesh, c1.geo, y.clone(), options=o)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    assert c1.mesh.info()["device_bytes"] == bytes_after_first  # plan and buffers reused


def test_sort_several_chunks(tp):
    """512 x 512 x 68 rays (> 2^24: two chunks) through a jittered Kuhn 6^3 mesh."""
    import torch
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(4, 900))
    mesh = tp.Mesh(verts, tets)
    g = W.ConeBeam(4.0, 8.0, 512, 512, 6.4 / 512, 6.4 / 512, W.uniform_angles(68))
    geo = tp.Geometry.from_cone(g)
    gen = torch.Generator(device="cuda").manual_seed(11)
    y = torch.rand(geo.shape + (4,), device="cuda", generator=gen)
    o_sort = _opts(tp, tp.SCATTER_SORT, 4, tile=(16, 8))
    a = tp.backward(mesh, geo, y, options=o_sort)
    b = tp.backward(mesh, geo, y, options=o_sort)
    ref = tp.backward(mesh, geo, y, options=_opts(tp, tp.SCATTER_ATOMIC, 4, tile=(16, 8)))
    flat = tp.backward(mesh, geo, y, options=tp.make_options(
        channels=4, tile=(16, 8), scatter=tp.SCATTER_ATOMIC, flags=tp.FLAG_ACC32))
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    assert torch.equal(a, b)
    # sampled tets against the oracle (y >= 0: the reference is its own scale).
    # ~10^5 segments reach each tet here; the sorted runs are summed with
    # compensation, the default atomic scatter is two-level here (FP32 sums of
    # one chunk merged into FP64), plain FP32 atomic sums drift (reported only).
    rng = np.random.default_rng(12)
    ts = rng.choice(tets.shape[0], 6, replace=False)
    want = oracle.backward_cone_subset(verts, tets, y.double().cpu().numpy().reshape(-1, 4), g, ts)
    idx = torch.tensor(ts, device="cuda")
    got = a[idx].double().cpu().numpy()
    got_atomic = ref[idx].double().cpu().numpy()
    got_flat = flat[idx].double().cpu().numpy()
    print(f"sort max rel {np.max(np.abs(got - want) / want):.2e}, "
          f"atomic two-level max rel {np.max(np.abs(got_atomic - want) / want):.2e}, "
          f"atomic FP32 max rel {np.max(np.abs(got_flat - want) / want):.2e}")
    assert np.all(np.abs(got - want) <= TOL["f32"] * want)
    assert np.all(np.abs(got_atomic - want) <= TOL["f32"] * want)


def test_sort_full_size_bench_workload(tp):
    import torch
    w = W.config2()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    mu = torch.tensor(w.mu, dtype=torch.float32, device="cuda")
    proj = tp.forward(mesh, geo, mu)
    o = _opts(tp, tp.SCATTER_SORT)
    a = tp.backward(mesh, geo, proj, options=o)
    b = tp.backward(mesh, geo, proj, options=o)
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    assert torch.equal(a, b)
    rng = np.random.default_rng(51)
    cen = W.tet_centroids(w.verts, w.tets)
    near = np.nonzero(np.linalg.norm(cen, axis=1) < 0.5)[0]
    ts = rng.choice(near, 4, replace=False)
    want = oracle.backward_cone_subset(w.verts, w.tets, proj.double().cpu().numpy().reshape(-1),
                                       w.geom, ts)
    got = a[torch.tensor(ts, device="cuda")].double().cpu().numpy()
    assert np.all(np.abs(got - want) <= TOL["f32"] * want)


def test_sort_rejected_where_unsupported(tp, c1):
    import torch
    y64 = torch.zeros(c1.geo.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(tp.TetprojError):  # plain FP64 path
        tp.backward(c1.mesh, c1.geo, y64,
                    options=tp.make_options(precision=tp.PLAIN_FP64, scatter=tp.SCATTER_SORT))
    src = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    src[:, 0] = 4.0
    dst = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(tp.TetprojError):  # explicit rays
        tp.backward_rays(c1.mesh, src, dst, torch.ones(4, device="cuda"),
                         options=_opts(tp, tp.SCATTER_SORT))
    with pytest.raises(tp.TetprojError):  # allocation-free call
        tp.backward_noalloc(c1.mesh, c1.geo, torch.zeros(c1.geo.shape, device="cuda"),
                            options=_opts(tp, tp.SCATTER_SORT))
    with pytest.raises(tp.TetprojError):  # batched launch
        tp.Batch([c1.mesh], [c1.geo], tiles=[(8, 8, 1, tp.SCATTER_SORT)])
