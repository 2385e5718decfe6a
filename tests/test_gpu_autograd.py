"""Differentiation through the projector (GPU).

TetProject.apply(mu) = A mu with backward g -> A^T g, the hand-written
backprojection (the exact adjoint of Eq. 2, i.e. Eq. 3).  Checked with
torch.autograd.gradcheck on a tiny case, against central finite differences of
the quadratic loss 0.5 |A mu - b|^2 on the config-4 mesh, and by running the
config-4 reconstruction (Adam, lr 1e-2, 100 iterations from mu = 0).  The
gradient of 0.5 |A mu - b|^2, A^T (A mu - b), is also compared with the
oracle's at sampled tets.
"""
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


def test_gradcheck_tiny(tp):
    import torch
    verts, tets = W.kuhn_cube(2)
    verts = W.jitter_interior(verts, tets, 2, W.rng_for(3, 7))
    mesh = tp.Mesh(verts, tets)
    geo = tp.Geometry(4.0, 8.0, 6, 5, 0.5, 0.5, W.uniform_angles(3))
    mu = torch.rand(mesh.nt, dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda m: tp.TetProject.apply(m, mesh, geo)
    assert torch.autograd.gradcheck(f, (mu,), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_finite_differences_config4(tp):
    """|FD - grad_k| <= 1e-6 (|grad_k| + 1e-3 max|grad|) on 32 tets, h = 1e-3, FP64,
    on the config-4 geometry (256 x 256 x 180 rays)."""
    import torch
    w = W.config4()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    rng = np.random.default_rng(41)
    mu0 = torch.tensor(rng.uniform(0, 1, mesh.nt), dtype=torch.float64, device="cuda")
    b = tp.forward(mesh, geo, torch.tensor(w.mu, dtype=torch.float64, device="cuda"))

    def loss(m):
        r = tp.TetProject.apply(m, mesh, geo) - b
        return 0.5 * (r * r).sum()

    mu = mu0.clone().requires_grad_(True)
    L = loss(mu)
    L.backward()
    grad = mu.grad.detach()
    gmax = float(grad.abs().max())
    # tets that rays actually cross (others have zero gradient and FD)
    hit = torch.nonzero(grad.abs() > 1e-3 * gmax).flatten().cpu().numpy()
    ks = rng.choice(hit, 32, replace=False)
    h = 1e-3
    with torch.no_grad():
        for k in ks:
            e = torch.zeros_like(mu0)
            e[k] = h
            fd = (float(loss(mu0 + e)) - float(loss(mu0 - e))) / (2 * h)
            gk = float(grad[k])
            assert abs(fd - gk) <= 1e-6 * (abs(gk) + 1e-3 * gmax), (k, fd, gk)


def test_reconstruction_config4(tp):
    """Config 4: b = A mu_true (FP64) + noise (sigma = 1% of max b); Adam on FP32 mu."""
    import torch
    w = W.config4()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    b64 = tp.forward(mesh, geo, torch.tensor(w.mu, dtype=torch.float64, device="cuda"))
    noise_rng = w.extra["noise_rng"]
    sigma = 0.01 * float(b64.max())
    b = (b64 + torch.tensor(noise_rng.normal(0, sigma, size=geo.shape), device="cuda")).float()
    mu = torch.zeros(mesh.nt, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([mu], lr=1e-2)
    true = torch.tensor(w.mu, dtype=torch.float32, device="cuda")
    losses = []
    for it in range(100):
        opt.zero_grad()
        r = tp.TetProject.apply(mu, mesh, geo) - b
        loss = 0.5 * (r * r).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    err0 = float(true.norm())
    err = float((mu.detach() - true).norm())
    floor = 0.5 * geo.nrays * sigma ** 2  # expected loss of the noise alone
    print(f"config4: loss {losses[0]:.1f} -> {losses[-1]:.1f} (noise floor ~{floor:.1f}), "
          f"|mu - mu_true| {err0:.2f} -> {err:.2f}")
    assert losses[-1] < 0.15 * losses[0], (losses[0], losses[-1], floor)
    assert err < 0.75 * err0, (err, err0)
    assert mesh.stats()["error"] == 0


@pytest.fixture(scope="module")
def c4_grad_ref():
    """Oracle side of the gradient check on the config-4 mesh and geometry.

    mu is supported on the ~420 tets within 0.08 of a seeded point (so that the
    oracle's A mu over all 11.8M rays is affordable: a_ij of the other tets is 0
    and each a_ij depends on its own tet only), b is seeded data on every ray.
    Returns r = A mu - b, and at 32 tets (16 in the support, 16 anywhere) the
    oracle's A^T r, A^T |r| and A^T A|mu| (the last two scale the tolerance:
    the backprojection's own error and the forward error carried into it)."""
    w = W.config4()
    rng = np.random.default_rng(43)
    cen = W.tet_centroids(w.verts, w.tets)
    c0 = rng.uniform(-0.4, 0.4, size=3)
    T = np.nonzero(np.linalg.norm(cen - c0, axis=1) < 0.08)[0]
    mu = np.zeros(w.tets.shape[0])
    mu[T] = rng.uniform(0.5, 1.5, size=T.size).astype(np.float32)
    b = rng.uniform(0.0, 0.2, size=w.geom.nrays).astype(np.float32).astype(np.float64)
    Amu = oracle.forward_cone(w.verts, w.tets[T], mu[T], w.geom)
    r = Amu - b
    sel = np.concatenate([rng.choice(T, 16, replace=False),
                          rng.choice(w.tets.shape[0], 16, replace=False)])
    y3 = np.stack([r, np.abs(r), Amu], axis=1)
    g = oracle.backward_cone_subset(w.verts, w.tets, y3, w.geom, sel)
    return dict(w=w, mu=mu, b=b, r=r, sel=sel, grad=g[:, 0], scale=g[:, 1] + g[:, 2], T=T)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_gradient_against_oracle_config4(tp, c4_grad_ref, prec):
    """The autograd gradient of 0.5 |A mu - b|^2 (forward kernel, then the
    hand-written backprojection of the residual) and the backprojection of the
    oracle's residual itself, at 32 tets, against the oracle's A^T (A mu - b):
    |g - g_ref| <= tau (A^T|r| + A^T A|mu|), tau = 1e-5 (FP32) / 1e-12 (FP64)."""
    import torch
    ref = c4_grad_ref
    w = ref["w"]
    dt = torch.float32 if prec == "f32" else torch.float64
    tau = 1e-5 if prec == "f32" else 1e-12
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    mu = torch.tensor(ref["mu"], dtype=dt, device="cuda", requires_grad=True)
    b = torch.tensor(ref["b"].reshape(geo.shape), dtype=dt, device="cuda")
    r = tp.TetProject.apply(mu, mesh, geo) - b
    loss = 0.5 * (r * r).sum()
    loss.backward()
    idx = torch.tensor(ref["sel"], device="cuda")
    got = mu.grad[idx].double().cpu().numpy()
    direct = tp.backward(mesh, geo, torch.tensor(ref["r"].reshape(geo.shape), dtype=dt,
                                                 device="cuda"))[idx].double().cpu().numpy()
    torch.cuda.synchronize()
    assert mesh.stats()["error"] == 0
    want, scale = ref["grad"], ref["scale"]
    for name, g in (("autograd", got), ("backward of the oracle residual", direct)):
        rel = np.abs(g - want) / scale
        print(f"C4 gradient {prec} {name}: max {rel.max():.3e} median {np.median(rel):.3e} "
              f"(relative to A^T|r| + A^T A|mu|)")
        assert np.all(np.abs(g - want) <= tau * scale), (name, rel.max())
    assert np.all(np.abs(want) > 0)
