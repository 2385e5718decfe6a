"""Reference iterative solvers over the oracle's projectors (test
infrastructure only; nothing in the product imports this module).

The paper poses reconstruction as the linear system A x = b (Eq. 1-3) and
solves it with OS-SART, 50 iterations over blocks of 20 projections (Sec. III-A,
image reconstruction); it also names CGLS among the usable algorithms
(Sec. II-A).  Both are written here from their textbook definitions, in FP64
numpy, over callables so that the same code runs on explicit dense matrices
(the pins in tests/test_oracle_solvers.py) and on the brute-force cone-beam
projectors of oracle/__init__.py.

OS-SART (ordered-subsets simultaneous algebraic reconstruction): for each
subset s of projections in turn,
    x <- x + lam * V_s^-1 A_s^T W_s (b_s - A_s x),
with W_s = diag(1 / row sums of A_s) (per ray; 0 for rays that miss) and
V_s = diag(column sums of A_s) (per tet; elements no ray of s crosses keep
their value), then optionally x <- max(x, 0).  One iteration = one pass over
all subsets.

CGLS (conjugate gradients on the normal equations A^T A x = A^T b), in the
usual form that never forms A^T A:
    r = b - A x, s = A^T r, p = s, gamma = |s|^2
    repeat: q = A p, alpha = gamma / |q|^2, x += alpha p, r -= alpha q,
            s = A^T r, gamma' = |s|^2, p = s + (gamma' / gamma) p.
"""
from __future__ import annotations

import numpy as np


def inverse_or_zero(v):
    """1 / v where v > 0, else 0 (weights of rays or tets with no intersection)."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    nz = v > 0
    out[nz] = 1.0 / v[nz]
    return out


def angle_blocks(nangles: int, block: int):
    """Subsets of consecutive projections: [0, block), [block, 2 block), ..."""
    return [np.arange(a, min(a + block, nangles)) for a in range(0, nangles, block)]


def ossart(forward_s, backward_s, b_s, x0, niter, lam=1.0, nonneg=True):
    """OS-SART.  forward_s[k](x) = A_k x, backward_s[k](y) = A_k^T y for
    subset k; b_s[k] = its measured rays.  Returns the iterate after `niter`
    passes over the subsets (and the list of iterates after each pass)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    nsub = len(forward_s)
    W = [inverse_or_zero(forward_s[k](np.ones_like(x))) for k in range(nsub)]
    V = [inverse_or_zero(backward_s[k](np.ones_like(b_s[k]))) for k in range(nsub)]
    history = []
    for _ in range(niter):
        for k in range(nsub):
            r = W[k] * (b_s[k] - forward_s[k](x))
            x = x + lam * V[k] * backward_s[k](r)
            if nonneg:
                x = np.maximum(x, 0.0)
        history.append(x.copy())
    return x, history


def cgls(forward, backward, b, x0, niter):
    """CGLS for min |A x - b|.  Returns (x, list of iterates)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = np.asarray(b, dtype=np.float64) - forward(x)
    s = backward(r)
    p = s.copy()
    gamma = float(np.dot(s, s))
    history = []
    for _ in range(niter):
        if gamma == 0.0:
            history.append(x.copy())
            continue
        q = forward(p)
        qq = float(np.dot(q, q))
        if qq == 0.0:
            history.append(x.copy())
            continue
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = backward(r)
        gamma_new = float(np.dot(s, s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        history.append(x.copy())
    return x, history


# ------------------------------------------------ cone-beam operators


def cone_subsets(geom, block: int):
    """(subset geometries, ray index arrays into the full scan) for blocks of
    `block` consecutive angles."""
    out = []
    per = geom.nu * geom.nv
    for idx in angle_blocks(geom.nangles, block):
        g = type(geom)(geom.dso, geom.dsd, geom.nu, geom.nv, geom.du, geom.dv,
                       np.asarray(geom.angles)[idx])
        rays = (idx[:, None] * per + np.arange(per)[None, :]).reshape(-1)
        out.append((g, rays))
    return out


def cone_operators(verts, tets, geom):
    """(A x, A^T y) on the full cone-beam scan with the oracle's projectors."""
    import oracle
    return (lambda x: oracle.forward_cone(verts, tets, x, geom),
            lambda y: oracle.backward_cone(verts, tets, y, geom))
