"""Batched persistent launch (GPU): problems of uneven size in one work-queue
launch per direction, through tetproj_batch_*.

* Reduced batched workload (jittered Kuhn meshes 3..12 cells per side,
  detectors 16..48 pixels per side, 3..12 angles, 4 channels), per-problem
  tiles of 32..256 rays: forward is bit-identical to the single-problem
  call with the same options (same walk, same arithmetic per ray), backward
  equal within tau * A^T|y| (atomic order differs), and sampled rays / tets
  match the oracle.
* CUDA graph: the forward + backward sequence captured once and replayed on
  new inputs written in place.
* Several rounds (more rays than one deferral-queue round holds), one mesh in
  two problems, a one-problem batch, argument errors.
* Autotuner: tune_batch picks per-problem tiles, and a second call is
  answered from its cache.
"""
import numpy as np
import pytest

import oracle
import workloads as W

from test_gpu_parity import TOL, check_rays, floor_abs, planar_reference

pytestmark = pytest.mark.gpu

SPECS = [(3, 16, 5), (8, 48, 9), (5, 24, 3), (12, 40, 7), (4, 32, 12), (6, 20, 4)]


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


@pytest.fixture(scope="module")
def probs(tp):
    ws = [W.config5_problem(k, n, N, na, channels=4) for k, (n, N, na) in enumerate(SPECS)]
    meshes = [tp.Mesh(w.verts, w.tets) for w in ws]
    geos = [tp.Geometry.from_cone(w.geom) for w in ws]
    return ws, meshes, geos


def _tiles(tp, threads, n):
    rows = {64: [(8, 8), (16, 4), (4, 16)], 128: [(16, 8), (8, 16), (32, 4)],
            0: [(8, 4), (16, 16), (4, 16), (32, 8), (16, 8), (8, 8)]}[threads]
    out = []
    for k in range(n):
        tu, tv = rows[k % len(rows)]
        out.append((tu, tv, tp.ORDER_MORTON if k % 2 == 0 else tp.ORDER_ROW,
                    tp.SCATTER_ATOMIC if (k // 2) % 2 == 0 else tp.SCATTER_WARP))
    return out


def _reference_channels(w, S, P, want, planar):
    """planar_reference per channel: (reference [n, C], rays without one)."""
    mu = w.mu.reshape(w.tets.shape[0], -1)
    out = np.array(want, dtype=np.float64).reshape(len(S), -1).copy()
    skipped = set()
    for c in range(mu.shape[1]):
        r = planar_reference(w.verts, w.tets, mu[:, c], S, P, out[:, c], planar)
        out[:, c] = r["want"]
        skipped |= set(r["skipped"])
    return out, sorted(skipped)


def _single_opts(tp, row, C):
    return tp.make_options(precision=tp.FILTERED, channels=C, tile=(row[0], row[1]),
                           order=row[2], scatter=row[3])


def _singles(tp, meshes, geos, mus, ys, tiles, C):
    fw, bw, sc = [], [], []
    for m, g, mu, y, row in zip(meshes, geos, mus, ys, tiles):
        o = _single_opts(tp, row, C)
        fw.append(tp.forward(m, g, mu, options=o))
        bw.append(tp.backward(m, g, y, options=o))
        sc.append(tp.backward(m, g, y.abs(), options=o))
    return fw, bw, sc


def _check_against_singles(tp, b, meshes, geos, tiles, C):
    import torch
    fw, bw, sc = _singles(tp, meshes, geos, b.mu, b.y, tiles, C)
    torch.cuda.synchronize()
    for k in range(len(meshes)):
        assert torch.equal(b.proj[k], fw[k]), f"problem {k}: batched forward differs"
        err = (b.mu_out[k].double() - bw[k].double()).abs()
        assert bool((err <= TOL["f32"] * sc[k].double() + 1e-30).all()), f"problem {k}"


@pytest.mark.parametrize("threads", [64, 128, 0])  # 0: a different tile per problem
def test_batch_matches_single_calls_and_oracle(tp, probs, threads):
    import torch
    ws, meshes, geos = probs
    tiles = _tiles(tp, threads, len(ws))
    for m in meshes:
        m.stats_reset()
    b = tp.Batch(meshes, geos, channels=4, tiles=tiles)
    for k, w in enumerate(ws):
        b.mu[k].copy_(torch.tensor(w.mu, dtype=torch.float32))
    b.forward()
    # rays the oracle flags as (nearly) inside a face plane carry y = 0 in the
    # backprojection: their split between the two sides is a convention
    planar_all = []
    for k, w in enumerate(ws):
        S, P = oracle.cone_rays(w.geom)
        planar_all.append(oracle.trace_rays(w.verts, w.tets, S, P, max_visits=2)[5])
        keep = torch.tensor(~planar_all[k], device="cuda", dtype=torch.float32)
        b.y[k].copy_(b.proj[k] * keep.reshape(geos[k].shape + (1,)))
    b.backward()
    torch.cuda.synchronize()
    _check_against_singles(tp, b, meshes, geos, tiles, 4)
    rng = np.random.default_rng(71 + threads)
    for k, w in enumerate(ws):
        assert meshes[k].stats()["error"] == 0
        # sampled rays against the oracle (exact references for face-plane rays)
        idx = np.sort(rng.choice(w.geom.nrays, min(64, w.geom.nrays), replace=False))
        S, P = oracle.cone_rays(w.geom, idx)
        want = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom, idx)
        scale = oracle.forward_cone(w.verts, w.tets, np.abs(w.mu), w.geom, idx)
        planar = planar_all[k][idx]
        ref, skipped = _reference_channels(w, S, P, want, planar)
        got = b.proj[k].reshape(-1, 4)[torch.tensor(idx, device="cuda")].double().cpu().numpy()
        fl = floor_abs("f32", w.verts, w.mu)
        for c in range(4):
            check_rays(f"batch problem {k} channel {c}", got[:, c], ref[:, c], scale[:, c],
                       TOL["f32"], fl, skipped, max_floor_frac=0.05)
        # sampled tets against the oracle's backprojection of the same y
        y = b.y[k].double().cpu().numpy().reshape(-1, 4)
        tets = rng.choice(w.tets.shape[0], min(8, w.tets.shape[0]), replace=False)
        wantb = oracle.backward_cone_subset(w.verts, w.tets, y, w.geom, tets)
        gotb = b.mu_out[k][torch.tensor(tets, device="cuda")].double().cpu().numpy()
        assert np.all(np.abs(gotb - wantb) <= TOL["f32"] * wantb), k
    b.close()


def test_batch_graph_capture_replay(tp, probs):
    import torch
    ws, meshes, geos = probs
    tiles = _tiles(tp, 64, len(ws))
    b = tp.Batch(meshes, geos, channels=4, tiles=tiles)
    gen = torch.Generator(device="cuda").manual_seed(5)
    for k in range(len(ws)):
        b.mu[k].uniform_(0, 1, generator=gen)
        b.y[k].uniform_(-1, 1, generator=gen)
    b.forward()
    b.backward()  # first calls outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.forward()
        b.backward()
    for it in range(2):
        for k in range(len(ws)):
            b.mu[k].uniform_(0, 1, generator=gen)
            b.y[k].uniform_(-1, 1, generator=gen)
        graph.replay()
        torch.cuda.synchronize()
        _check_against_singles(tp, b, meshes, geos, tiles, 4)
    del graph
    b.close()


def test_batch_several_rounds_and_shared_mesh(tp):
    """One problem of 512 x 512 x 136 rays (> 2^25, two rounds of the batch's
    deferral queue) and a second problem on the same mesh, one channel."""
    import torch
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(4, 900))
    mu = W.rng_for(4, 901).uniform(0, 1, tets.shape[0])
    mesh = tp.Mesh(verts, tets)
    g_big = W.ConeBeam(4.0, 8.0, 512, 512, 6.4 / 512, 6.4 / 512, W.uniform_angles(136))
    g_small = W.ConeBeam(4.0, 8.0, 24, 20, 0.3, 0.3, W.uniform_angles(5))
    assert g_big.nrays > 2 ** 25
    geos = [tp.Geometry.from_cone(g_big), tp.Geometry.from_cone(g_small)]
    tiles = [(16, 8, tp.ORDER_MORTON, tp.SCATTER_ATOMIC), (8, 16, tp.ORDER_ROW, tp.SCATTER_WARP)]
    mesh.stats_reset()
    b = tp.Batch([mesh, mesh], geos, channels=1, tiles=tiles)
    for k in range(2):
        b.mu[k].copy_(torch.tensor(mu, dtype=torch.float32))
        b.y[k].uniform_(0, 1)
    b.forward()
    b.backward()
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    _check_against_singles(tp, b, [mesh, mesh], geos, tiles, 1)
    rng = np.random.default_rng(81)
    idx = np.sort(rng.choice(g_big.nrays, 64, replace=False))
    want = oracle.forward_cone(verts, tets, mu, g_big, idx)
    scale = oracle.forward_cone(verts, tets, np.abs(mu), g_big, idx)
    got = b.proj[0].reshape(-1)[torch.tensor(idx, device="cuda")].double().cpu().numpy()
    S, P = oracle.cone_rays(g_big, idx)
    _, _, _, _, _, planar = oracle.trace_rays(verts, tets, S, P, max_visits=2)
    check_rays("batch several rounds", got, want, scale, TOL["f32"], floor_abs("f32", verts, mu),
               np.nonzero(planar)[0], max_floor_frac=0.05)
    # a one-problem batch
    b1 = tp.Batch([mesh], geos[1:], channels=1, tiles=tiles[1:])
    b1.mu[0].copy_(b.mu[1])
    b1.forward()
    torch.cuda.synchronize()
    assert torch.equal(b1.proj[0], b.proj[1])
    b.close()
    b1.close()


def test_batch_dense_two_level_accumulation(tp):
    """A dense 4-channel problem (1296 tets, 512 x 512 x 34 rays: ~10^5
    segments per tet; backprojection rounds cut inside the dense problem) through the batched launch and
    a single call: both backprojections use two-level accumulation (FP32
    reductions merged into FP64 after every round / chunk) and meet the FP32
    target on sampled tets against the oracle's FP64 sums."""
    import torch
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(4, 900))
    mesh = tp.Mesh(verts, tets)
    g = W.ConeBeam(4.0, 8.0, 512, 512, 6.4 / 512, 6.4 / 512, W.uniform_angles(34))
    geo = tp.Geometry.from_cone(g)
    b = tp.Batch([mesh], [geo], channels=4, tiles=[(16, 8, tp.ORDER_MORTON, tp.SCATTER_ATOMIC)])
    gen = torch.Generator(device="cuda").manual_seed(17)
    b.y[0].copy_(torch.rand(b.y[0].shape, device="cuda", generator=gen))
    b.backward()
    single = tp.backward(mesh, geo, b.y[0], options=tp.make_options(channels=4, tile=(16, 8)))
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    rng = np.random.default_rng(19)
    ts = rng.choice(tets.shape[0], 5, replace=False)
    want = oracle.backward_cone_subset(verts, tets, b.y[0].double().cpu().numpy().reshape(-1, 4), g, ts)
    idx = torch.tensor(ts, device="cuda")
    for got in (b.mu_out[0][idx], single[idx]):
        got = got.double().cpu().numpy()
        assert np.all(np.abs(got - want) <= TOL["f32"] * want), np.max(np.abs(got - want) / want)
    b.close()


def test_batch_argument_errors(tp, probs):
    ws, meshes, geos = probs
    with pytest.raises(tp.TetprojError):  # fewer than 32 rays per tile
        tp.Batch(meshes[:2], geos[:2], tiles=[(8, 8, 1, 0), (4, 4, 1, 0)])
    with pytest.raises(tp.TetprojError):  # more than 256 rays per tile
        tp.Batch(meshes[:1], geos[:1], tiles=[(32, 16, 1, 0)])
    with pytest.raises(tp.TetprojError):  # not a power of two
        tp.Batch(meshes[:1], geos[:1], tiles=[(12, 8, 1, 0)])
    with pytest.raises(tp.TetprojError):
        tp.Batch(meshes[:1], geos[:1], channels=3)
    with pytest.raises(ValueError):
        tp.Batch(meshes[:2], geos[:1])


def test_autotune_batch_and_cache(tp, probs, tmp_path):
    import torch
    from paper_1908_06909_gb300 import autotune as A
    ws, meshes, geos = probs
    cache = A.Cache(str(tmp_path / "tune.json"), device=torch.cuda.get_device_name(),
                    version=tp.version())
    choices = A.tune_batch(tp, meshes[:3], geos[:3], channels=4, cache=cache, reps=1)
    assert len(choices) == 3
    for c in choices:
        assert c.tile_u * c.tile_v >= 32
    # answered from the cache: no measurement
    orig = A.gpu_measure
    A.gpu_measure = lambda *a, **k: (_ for _ in ()).throw(AssertionError("measured again"))
    try:
        again = A.tune_batch(tp, meshes[:3], geos[:3], channels=4,
                             cache=A.Cache(str(tmp_path / "tune.json"),
                                           device=torch.cuda.get_device_name(),
                                           version=tp.version()))
    finally:
        A.gpu_measure = orig
    assert again == choices
    b = tp.Batch(meshes[:3], geos[:3], channels=4, tiles=[c.row() for c in choices])
    for k in range(3):
        b.mu[k].copy_(torch.tensor(ws[k].mu, dtype=torch.float32))
    b.forward()
    torch.cuda.synchronize()
    for k in range(3):
        single = tp.forward(meshes[k], geos[k], b.mu[k], options=_single_opts(tp, choices[k].row(), 4))
        assert torch.equal(b.proj[k], single)
    b.close()


def test_batch_bounded_wait_times_out_and_recovers(tp, probs):
    """The persistent kernel's inter-warp waits are bounded.  Made to wait for a
    value no warp writes (a test-only setting), every wait runs out after 16
    polls: the launch still completes, the statistics report
    TETPROJ_ERR_TIMEOUT, and the next call with the default bound succeeds and
    equals the single-problem calls."""
    import torch
    ws, meshes, geos = probs
    ms, gs, wk = meshes[:3], geos[:3], ws[:3]
    b = tp.Batch(ms, gs, channels=4)
    for k in range(3):
        b.mu[k].copy_(torch.tensor(wk[k].mu, dtype=torch.float32))
    for m in ms:
        m.stats_reset()
    b.set_wait(max_polls=16, never_satisfied=True)
    b.forward()
    torch.cuda.synchronize()
    errs = [m.stats()["error"] for m in ms]
    assert tp._lib.ERR_TIMEOUT in errs and all(e in (0, tp._lib.ERR_TIMEOUT) for e in errs), errs
    with pytest.raises(tp.TetprojError):
        b.set_wait(max_polls=-1)
    b.set_wait()  # the default bound
    for m in ms:
        m.stats_reset()
    b.proj[0].zero_()
    b.forward()
    torch.cuda.synchronize()
    assert all(m.stats()["error"] == 0 for m in ms)
    for k in range(3):
        single = tp.forward(ms[k], gs[k], b.mu[k], options=tp.make_options(channels=4))
        assert torch.equal(single, b.proj[k])
    b.close()
