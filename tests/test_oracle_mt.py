"""Pins of the reference of the paper's walk (oracle/mt.c): in FP64 on generic
rays it must reproduce the plain definition (brute-force clipping, oracle.c,
an independent computation) and finish every ray; a ray that misses the mesh
gives 0."""
import numpy as np

import oracle
import workloads as W


def test_mt_fp64_generic_rays_equal_definition():
    n = 4
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(6, 11))
    mu = W.rng_for(6, 12).uniform(0, 1, tets.shape[0])
    S, P = W.random_rays_through_box(400, W.rng_for(6, 13))
    got, st = oracle.mt_forward_rays(verts, tets, mu, S, P, "f64")
    want = oracle.forward_rays(verts, tets, mu, S, P)
    scale = oracle.forward_rays(verts, tets, np.abs(mu), S, P)
    assert np.all(st == 0)
    assert np.all(np.abs(got - want) <= 1e-12 * scale + 1e-15)
    assert (want > 0).sum() > 300


def test_mt_fp32_close_to_definition_on_generic_rays():
    n = 4
    verts, tets = W.kuhn_cube(n)
    verts = W.jitter_interior(verts, tets, n, W.rng_for(6, 14))
    mu = W.rng_for(6, 15).uniform(0, 1, tets.shape[0]).astype(np.float32).astype(np.float64)
    S, P = W.random_rays_through_box(400, W.rng_for(6, 16))
    got, st = oracle.mt_forward_rays(verts, tets, mu, S, P, "f32")
    want = oracle.forward_rays(verts, tets, mu, S, P)
    scale = oracle.forward_rays(verts, tets, np.abs(mu), S, P)
    ok = st == 0
    assert ok.mean() > 0.99
    assert np.all(np.abs(got - want)[ok] <= 1e-4 * scale[ok] + 1e-6)


def test_mt_miss_is_zero():
    verts, tets = W.kuhn_cube(2)
    S = np.array([[4.0, 3.0, 0.0]])
    P = np.array([[-4.0, 3.0, 0.0]])
    got, st = oracle.mt_forward_rays(verts, tets, np.ones(tets.shape[0]), S, P, "f64")
    assert got[0] == 0.0 and st[0] == 0
