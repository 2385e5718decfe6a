"""Differentiation through the projector (GPU).

TetProject.apply(mu) = A mu with backward g -> A^T g, the hand-written
backprojection (the exact adjoint of Eq. 2, i.e. Eq. 3).  Checked with
torch.autograd.gradcheck on a tiny case, against central finite differences of
the quadratic loss 0.5 |A mu - b|^2 on the config-4 mesh, and by running the
config-4 reconstruction (Adam, lr 1e-2, 100 iterations from mu = 0).
"""
import numpy as np
import pytest

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
    """|FD - grad_k| <= 1e-6 (|grad_k| + 1e-3 max|grad|) on 32 tets, h = 1e-3, FP64."""
    import torch
    w = W.config4(nangles=12)
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
