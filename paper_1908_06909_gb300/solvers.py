"""Iterative reconstruction on the GPU projectors.

The paper reconstructs with OS-SART, 50 iterations over blocks of 20
projections (Sec. III-A), and names CGLS among the algorithms the projectors
serve (Sec. II-A): every such algorithm needs only A x and A^T y (Eq. 2, 3).
Here both run on ``tetproj_forward`` / ``tetproj_backward`` (float32 tensors:
the filtered path; float64: the plain FP64 path); the O(n) vector updates
between projections are torch element-wise operations on the same device and
stream (under 1% of an iteration's time: each iteration projects every ray
twice).

OS-SART, per subset s of projections in turn:
    x <- x + lam * V_s^-1 A_s^T W_s (b_s - A_s x),   then x <- max(x, 0)
with W_s = 1 / (A_s 1) per ray and V_s = A_s^T 1 per tet (0 where nothing is
crossed; such tets keep their value).  Subsets are blocks of consecutive
projections (the paper gives the block size, not the order).

CGLS: conjugate gradients on A^T A x = A^T b without forming A^T A.
"""
from __future__ import annotations

import numpy as np

from . import Geometry, backward, forward


def _safe_inv(t):
    import torch
    out = torch.zeros_like(t)
    nz = t > 0
    out[nz] = 1.0 / t[nz]
    return out


class OSSART:
    """OS-SART on a cone-beam scan split into blocks of `block` projections.

    b: measured projections [nangles, nv, nu] (device tensor; its dtype picks
    the path).  The subset geometries and the weights W_s, V_s are computed
    once here (one forward and one backward projection of ones per subset)."""

    def __init__(self, mesh, geo: Geometry, b, block: int = 20, lam: float = 1.0,
                 nonneg: bool = True, options=None):
        import torch
        self.mesh, self.lam, self.nonneg, self.options = mesh, lam, nonneg, options
        self.dtype = b.dtype
        ang = np.asarray(geo.angles, dtype=np.float64)
        self.subsets = []
        for a0 in range(0, geo.nangles, block):
            idx = np.arange(a0, min(a0 + block, geo.nangles))
            g = Geometry(geo.dso, geo.dsd, geo.nu, geo.nv, geo.du, geo.dv, ang[idx])
            bs = b[a0:a0 + len(idx)].contiguous()
            ones_x = torch.ones(mesh.nt, dtype=self.dtype, device=b.device)
            W = _safe_inv(forward(mesh, g, ones_x, options=options))
            V = _safe_inv(backward(mesh, g, torch.ones_like(bs), options=options))
            self.subsets.append((g, bs, W, V))

    def iterate(self, x, niter: int = 1):
        """`niter` passes over all subsets, in place on x; returns x."""
        for _ in range(niter):
            for g, bs, W, V in self.subsets:
                r = (bs - forward(self.mesh, g, x, options=self.options)) * W
                x += self.lam * V * backward(self.mesh, g, r, options=self.options)
                if self.nonneg:
                    x.clamp_(min=0)
        return x


def ossart(mesh, geo: Geometry, b, niter: int = 50, block: int = 20, lam: float = 1.0,
           nonneg: bool = True, x0=None, options=None):
    """OS-SART reconstruction (defaults: the paper's 50 iterations, blocks of 20)."""
    import torch
    x = torch.zeros(mesh.nt, dtype=b.dtype, device=b.device) if x0 is None else x0.clone()
    return OSSART(mesh, geo, b, block, lam, nonneg, options).iterate(x, niter)


def cgls(mesh, geo: Geometry, b, niter: int = 20, x0=None, options=None, callback=None):
    """CGLS for min |A x - b|; callback(k, x) after each iteration.

    Every scalar stays on the device (no host synchronisation inside the
    loop, so the iterations queue back to back and can be captured in a CUDA
    graph): a zero step length or direction, where the textbook loop would
    stop, makes the remaining iterations leave x unchanged instead."""
    import torch
    x = torch.zeros(mesh.nt, dtype=b.dtype, device=b.device) if x0 is None else x0.clone()
    r = b - forward(mesh, geo, x, options=options)
    s = backward(mesh, geo, r, options=options)
    p = s.clone()
    gamma = torch.dot(s, s)
    zero = torch.zeros((), dtype=b.dtype, device=b.device)
    for k in range(niter):
        q = forward(mesh, geo, p, options=options)
        qq = torch.dot(q.reshape(-1), q.reshape(-1))
        alpha = torch.where(qq > 0, gamma / torch.where(qq > 0, qq, 1), zero)
        x += alpha * p
        r -= alpha * q
        s = backward(mesh, geo, r, options=options)
        gamma_new = torch.dot(s, s)
        beta = torch.where(gamma > 0, gamma_new / torch.where(gamma > 0, gamma, 1), zero)
        p = s + beta * p
        gamma = gamma_new
        if callback is not None:
            callback(k, x)
    return x
