"""tetproj_backward_noalloc against tetproj_backward and the oracle (GPU).

Some callers cannot call cudaMalloc when they backproject (their device memory
is owned by another allocator, or they must not pay cudaMalloc's implicit
synchronisation), so the library offers a backprojection whose scratch is a
fixed device array inside the library.  These tests call it through the C ABI,
twice in a row where it matters (the array keeps the previous call's
contents, so the second call checks that everything that must start at zero is
cleared), and compare each result with tetproj_backward within the parity
tolerance of the GPU tests: per tet |x_noalloc - x_backward| <= tau * sum_j
a_ij |y_j| (tau = 1e-12 plain FP64, 1e-5 filtered FP32).  Covered: both
precisions; more rays than the fixed deferral queue holds (several chunks
reuse it); C = 4 with FP32 atomics and with warp-aggregated atomics; a dense
C = 4 problem (two-level accumulation inside the fixed array) against the
oracle's FP64 sums; the size limit and the options it does not offer.
They run alone or after the other tests.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TAU = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def tp():
    import torch
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    import paper_1908_06909_gb300 as tp
    return tp


def _compare(tp, mesh, geo, y, tau, options=None):
    import torch
    ref = tp.backward(mesh, geo, y, options=options)
    mag = tp.backward(mesh, geo, y.abs(), options=options)
    out = tp.backward_noalloc(mesh, geo, y, options=options)
    torch.cuda.synchronize()
    err = (out.double() - ref.double()).abs()
    bound = tau * mag.double() + 1e-300
    assert bool((err <= bound).all()), float((err / bound).max())
    assert float(mag.max()) > 0
    return out


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_backward_noalloc_matches_backward(tp, prec):
    import torch
    dt = torch.float64 if prec == "f64" else torch.float32
    w = W.config1()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    gen = torch.Generator("cuda").manual_seed(17)
    for call in range(2):
        y = torch.rand(geo.shape, dtype=dt, device="cuda", generator=gen)
        if call == 1:
            y = y * 3.0 - 1.0  # different values and signs on the second call
        _compare(tp, mesh, geo, y, TAU[prec])
    assert mesh.stats()["error"] == 0


@pytest.mark.parametrize("channels,scatter", [(1, "atomic"), (4, "atomic"), (4, "warp")])
def test_backward_noalloc_several_queue_chunks(tp, channels, scatter):
    """128 x 128 x 32 = 524,288 rays: more than the fixed 2^18-entry deferral
    queue, so the walk runs in chunks that reuse it."""
    import torch
    w = W.config1(det=128, pitch=0.05)
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    assert geo.nrays > 2 ** 18
    sc = tp.SCATTER_WARP if scatter == "warp" else tp.SCATTER_ATOMIC
    opts = tp.make_options(channels=channels, scatter=sc)
    shape = geo.shape + ((4,) if channels == 4 else ())
    gen = torch.Generator("cuda").manual_seed(23)
    for call in range(2):
        y = torch.rand(shape, dtype=torch.float32, device="cuda", generator=gen) - 0.25 * call
        _compare(tp, mesh, geo, y, TAU["f32"], opts)
    assert mesh.stats()["error"] == 0


def test_backward_noalloc_dense_two_level_against_oracle(tp):
    """A dense 4-channel problem (1296 tets, 512 x 512 x 34 rays, ~10^5
    segments per tet): the default accumulation is two-level (FP32 reductions
    merged into FP64 after every chunk), here inside the fixed array; sampled
    tets meet the FP32 target against the oracle's FP64 sums."""
    import torch
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(4, 900))
    mesh = tp.Mesh(verts, tets)
    g = W.ConeBeam(4.0, 8.0, 512, 512, 6.4 / 512, 6.4 / 512, W.uniform_angles(34))
    geo = tp.Geometry.from_cone(g)
    opts = tp.make_options(channels=4, tile=(16, 8))
    gen = torch.Generator("cuda").manual_seed(29)
    y = torch.rand(geo.shape + (4,), dtype=torch.float32, device="cuda", generator=gen)
    out = _compare(tp, mesh, geo, y, TAU["f32"], opts)
    rng = np.random.default_rng(31)
    ts = rng.choice(tets.shape[0], 8, replace=False)
    want = oracle.backward_cone_subset(verts, tets, y.double().cpu().numpy().reshape(-1, 4), g, ts)
    got = out[torch.tensor(ts, device="cuda")].double().cpu().numpy()
    assert np.all(np.abs(got - want) <= TAU["f32"] * want), np.max(np.abs(got - want) / want)
    assert mesh.stats()["error"] == 0


def test_backward_noalloc_limits(tp):
    """Beyond the fixed accumulator (plain FP64, C = 4: 56^3 cells = 1,053,696
    tets x 32 bytes > 32 MB) the call returns TETPROJ_ERR_TOO_LARGE; the
    sort-and-reduce scatter is refused with TETPROJ_ERR_ARG.  Both are decided
    before any GPU work."""
    import torch
    verts, tets = W.kuhn_cube(56)
    mesh = tp.Mesh(verts, tets)
    assert mesh.nt * 4 * 8 > 32 * 1024 * 1024
    g = W.ConeBeam(4.0, 8.0, 8, 8, 0.8, 0.8, W.uniform_angles(2))
    geo = tp.Geometry.from_cone(g)
    y = torch.ones(geo.shape + (4,), dtype=torch.float64, device="cuda")
    with pytest.raises(tp.TetprojError) as e:
        tp.backward_noalloc(mesh, geo, y, options=tp.make_options(precision=tp.PLAIN_FP64, channels=4))
    assert e.value.code == tp._lib.ERR_TOO_LARGE
    small = W.config1(n_cells=4, det=8, pitch=0.8, nangles=2)
    m2 = tp.Mesh(small.verts, small.tets)
    g2 = tp.Geometry.from_cone(small.geom)
    with pytest.raises(tp.TetprojError) as e:
        tp.backward_noalloc(m2, g2, torch.ones(g2.shape, device="cuda"),
                            options=tp.make_options(scatter=tp.SCATTER_SORT))
    assert e.value.code == tp._lib.ERR_ARG
