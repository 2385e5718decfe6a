"""Entry search (GPU): the BVH and the paper's R*-tree give the oracle's
first tet; the R*-tree entry leaves the forward projection bit-identical;
calls without an R*-tree variant reject the flag; and the split of a single
1024 x 1024 projection into entry search ("initialization") and propagation
over regular meshes of growing size, as in the paper's performance figure
(printed; recorded in the design notes)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    return tp


def test_entry_tet_matches_oracle(tp):
    import torch
    n = 8
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(7, 2))
    geom = W.ConeBeam(4.0, 8.0, 40, 32, 0.2, 0.2, W.uniform_angles(12) + 0.07)
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry.from_cone(geom)
    e_bvh = tp.entry(mesh, geo).cpu().numpy().reshape(-1)
    e_rs = tp.entry(mesh, geo, options=tp.make_options(flags=tp.FLAG_RSTAR_ENTRY)).cpu().numpy().reshape(-1)
    S, P = oracle.cone_rays(geom)
    tt, lo, hi, cnt, margin, planar = oracle.trace_rays(verts, tets, S, P, max_visits=4)
    want = np.where(cnt > 0, tt[:, 0], -1)
    ok = ~planar
    assert ok.mean() > 0.99
    assert np.array_equal(e_bvh[ok], want[ok])
    assert np.array_equal(e_rs, e_bvh)
    assert (want >= 0).sum() > 0.5 * want.size


def test_rstar_entry_forward_identical(tp):
    import torch
    n = 16
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(7, 3))
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry(4.0, 8.0, 64, 64, 0.1, 0.1, W.uniform_angles(8))
    mu = torch.rand(mesh.nt, device="cuda")
    a = tp.forward(mesh, geo, mu)
    mesh.stats_reset()
    b = tp.forward(mesh, geo, mu, options=tp.make_options(flags=tp.FLAG_RSTAR_ENTRY))
    st = mesh.stats()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert st["error"] == 0 and st["bvh_faces"] > 0


def test_rstar_flag_rejected_where_unsupported(tp):
    import torch
    verts, tets = W.kuhn_cube(3)
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry(4.0, 8.0, 16, 16, 0.4, 0.4, W.uniform_angles(2))
    o = tp.make_options(flags=tp.FLAG_RSTAR_ENTRY)
    with pytest.raises(tp.TetprojError):
        tp.backward(mesh, geo, torch.ones(geo.shape, device="cuda"), options=o)
    with pytest.raises(tp.TetprojError):
        tp.forward(mesh, geo, torch.ones(mesh.nt, dtype=torch.float64, device="cuda"),
                   options=tp.make_options(precision=tp.PLAIN_FP64, flags=tp.FLAG_RSTAR_ENTRY))
    with pytest.raises(tp.TetprojError):
        tp.forward(mesh, geo, torch.ones((mesh.nt, 4), device="cuda"),
                   options=tp.make_options(channels=4, flags=tp.FLAG_RSTAR_ENTRY))
    with pytest.raises(tp.TetprojError):  # unknown flag
        tp.forward(mesh, geo, torch.ones(mesh.nt, device="cuda"), options=tp.make_options(flags=8))


def _time(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def test_initialization_vs_propagation_sweep(tp):
    """One 1024^2 projection of regular Kuhn meshes, n = 8..128 cells per side."""
    import torch
    geo = tp.Geometry(4.0, 8.0, 1024, 1024, 0.00625, 0.00625, np.array([0.3]))
    rows = []
    for n in (8, 16, 32, 64, 96, 128):
        verts, tets = W.kuhn_cube(n)
        mesh = tp.Mesh(verts, tets)
        mu = torch.ones(mesh.nt, device="cuda")
        rs = tp.make_options(flags=tp.FLAG_RSTAR_ENTRY)
        t_init = _time(lambda: tp.entry(mesh, geo))
        t_init_rs = _time(lambda: tp.entry(mesh, geo, options=rs))
        t_fwd = _time(lambda: tp.forward(mesh, geo, mu))
        t_fwd_rs = _time(lambda: tp.forward(mesh, geo, mu, options=rs))
        a, b = tp.forward(mesh, geo, mu), tp.forward(mesh, geo, mu, options=rs)
        assert torch.equal(a, b)
        info = mesh.info()
        rows.append((n, mesh.nt, info["nboundary"], t_init, t_fwd - t_init, t_init_rs,
                     t_fwd_rs - t_init_rs))
        del mesh
    print("\n  n   tets        boundary  init BVH ms  propagate ms  init R* ms  propagate(R*) ms")
    for r in rows:
        print(f"{r[0]:4d} {r[1]:10d} {r[2]:9d} {r[3]:11.3f} {r[4]:13.3f} {r[5]:11.3f} {r[6]:14.3f}")
    # propagation grows with the edge length, the entry search stays small
    assert rows[-1][4] > rows[0][4]
