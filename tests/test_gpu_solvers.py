"""Iterative solvers on the GPU projectors (OS-SART, CGLS), GPU.

* FP64 parity: iterates of OS-SART (blocks of 5 of 20 projections) and of
  CGLS on a jittered Kuhn 6^3 mesh agree with the oracle's solvers
  (oracle/solvers.py over the brute-force projectors) to ~1e-12 relative per
  projection, compounded over the iterations (tolerance 1e-9).
* FP32 reconstruction: the paper's OS-SART setting (50 iterations, blocks of
  20 projections, 100 projections) on a jittered Kuhn 12^3 phantom with a
  32^2 detector recovers the phantom (relative error below 5%) and CGLS
  reduces the residual monotonically in its normal-equations norm.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import solvers as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


@pytest.fixture(scope="module")
def small():
    n = 6
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(5, 1))
    cen = W.tet_centroids(verts, tets)
    x_true = 0.3 + (np.linalg.norm(cen, axis=1) < 0.6) * 0.7
    # angles offset from multiples of 90 degrees: no ray near a face plane
    geom = W.ConeBeam(4.0, 8.0, 12, 10, 0.5, 0.5, W.uniform_angles(20) + 0.1)
    S, P = oracle.cone_rays(geom)
    planar = oracle.trace_rays(verts, tets, S, P, max_visits=2)[5]
    assert not planar.any()
    b = oracle.forward_cone(verts, tets, x_true, geom)
    return verts, tets, geom, x_true, b


def test_ossart_fp64_matches_oracle(tp, small):
    import torch
    from paper_1908_06909_gb300 import solvers
    verts, tets, geom, x_true, b = small
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry.from_cone(geom)
    bt = torch.tensor(b.reshape(geo.shape), dtype=torch.float64, device="cuda")
    sol = solvers.OSSART(mesh, geo, bt, block=5)
    x = torch.zeros(mesh.nt, dtype=torch.float64, device="cuda")
    subs = OS.cone_subsets(geom, 5)
    fs = [(lambda x, g=g: oracle.forward_cone(verts, tets, x, g)) for g, _ in subs]
    bs = [(lambda y, g=g: oracle.backward_cone(verts, tets, y, g)) for g, _ in subs]
    _, hist = OS.ossart(fs, bs, [b[r] for _, r in subs], np.zeros(tets.shape[0]), 3)
    for k in range(3):
        sol.iterate(x, 1)
        got = x.cpu().numpy()
        rel = np.linalg.norm(got - hist[k]) / np.linalg.norm(hist[k])
        print(f"OS-SART iteration {k + 1}: rel diff {rel:.2e}")
        assert rel < 1e-9


def test_cgls_fp64_matches_oracle(tp, small):
    import torch
    from paper_1908_06909_gb300 import solvers
    verts, tets, geom, x_true, b = small
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry.from_cone(geom)
    bt = torch.tensor(b.reshape(geo.shape), dtype=torch.float64, device="cuda")
    got = []
    solvers.cgls(mesh, geo, bt.reshape(-1).reshape(geo.shape), niter=4,
                 callback=lambda k, x: got.append(x.cpu().numpy().copy()))
    f, bk = OS.cone_operators(verts, tets, geom)
    _, hist = OS.cgls(f, bk, b, np.zeros(tets.shape[0]), 4)
    for k in range(4):
        rel = np.linalg.norm(got[k] - hist[k]) / np.linalg.norm(hist[k])
        print(f"CGLS iteration {k + 1}: rel diff {rel:.2e}")
        assert rel < 1e-9


def test_ossart_fp32_paper_setting_reconstructs(tp):
    import torch
    from paper_1908_06909_gb300 import solvers
    n = 12
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(5, 2))
    cen = W.tet_centroids(verts, tets)
    x_true = W.phantom_at(cen, *W.phantom_params(W.rng_for(5, 3)))
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry(4.0, 8.0, 32, 32, 0.2, 0.2, W.uniform_angles(100))
    xt = torch.tensor(x_true, dtype=torch.float32, device="cuda")
    b = tp.forward(mesh, geo, xt)
    x = solvers.ossart(mesh, geo, b, niter=50, block=20)
    err = float((x - xt).norm() / xt.norm())
    print(f"OS-SART 50 it, 5 blocks of 20: relative error {err:.3e}")
    assert err < 0.05
    assert mesh.stats()["error"] == 0


def test_cgls_fp32_normal_residual_decreases(tp):
    import torch
    from paper_1908_06909_gb300 import solvers
    n = 10
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(5, 4))
    cen = W.tet_centroids(verts, tets)
    x_true = W.phantom_at(cen, *W.phantom_params(W.rng_for(5, 5)))
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry(4.0, 8.0, 32, 32, 0.2, 0.2, W.uniform_angles(60))
    xt = torch.tensor(x_true, dtype=torch.float32, device="cuda")
    b = tp.forward(mesh, geo, xt)
    norms = []

    def cb(k, x):
        r = b - tp.forward(mesh, geo, x)
        norms.append(float(tp.backward(mesh, geo, r).norm()))

    x = solvers.cgls(mesh, geo, b, niter=15, callback=cb)
    assert all(norms[k + 1] < norms[k] * 1.5 for k in range(len(norms) - 1))
    assert norms[-1] < 0.05 * norms[0]
    assert float((x - xt).norm() / xt.norm()) < 0.25


def test_cgls_no_host_sync(tp, small):
    """CGLS keeps its scalars on the device: no torch operation in its loop
    synchronises with the host (after a first call has allocated the mesh's
    workspace), and the result equals the oracle's iterates as above."""
    import torch
    from paper_1908_06909_gb300 import solvers
    verts, tets, geom, x_true, b = small
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry.from_cone(geom)
    bt = torch.tensor(b.reshape(geo.shape), dtype=torch.float64, device="cuda")
    solvers.cgls(mesh, geo, bt, niter=1)
    torch.cuda.synchronize()
    torch.cuda.set_sync_debug_mode("error")
    try:
        x = solvers.cgls(mesh, geo, bt, niter=4)
    finally:
        torch.cuda.set_sync_debug_mode("default")
    f, bk = OS.cone_operators(verts, tets, geom)
    _, hist = OS.cgls(f, bk, b, np.zeros(tets.shape[0]), 4)
    assert np.linalg.norm(x.cpu().numpy() - hist[3]) <= 1e-9 * np.linalg.norm(hist[3])
