"""Seeded synthetic workloads for the tetrahedral-mesh projectors.

This module only *generates inputs*: meshes, attenuation fields, cone-beam
parameters and explicit rays.  It holds none of the projector arithmetic
(no chord lengths, no traversal, no predicates), so both the CPU oracle and
the CUDA path can consume the same arrays without sharing method code.

The paper times its kernels on voxel grids split into tetrahedra (Sec. III-D,
performance figures) and shows precision failures on a Delaunay mesh with
badly shaped tets (Sec. III-C, floating point errors).  Neither mesh ships with the paper, so
the stand-ins are Kuhn (Freudenthal) splits of the cube [-1, 1]^3:

* ``kuhn_cube(n)``: n^3 cells, each split into 6 tets along its v000->v111
  diagonal, the same split in every cell (a conforming triangulation).
* ``jitter_interior``: interior vertices moved by U[-0.2h, 0.2h] per axis.
* ``cubic_map``: x -> sign(x)|x|^3 per axis, spacing ratio ~3e3 at n=64.

Seeds follow ``SEED_BASE + config_index`` with NumPy's PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 190806909


def rng_for(config_index: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for a workload; ``stream`` separates independent draws."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + config_index, stream]))


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def grid_coords(n: int) -> np.ndarray:
    """The n+1 grid abscissae of [-1, 1]: (2i - n)/n, exact at -1, 0 (n even), 1."""
    i = np.arange(n + 1, dtype=np.float64)
    return (2.0 * i - n) / n


def kuhn_cube(n: int):
    """Kuhn split of [-1,1]^3 into n^3 cells x 6 tets.

    Vertex (i, j, k) has index (k*(n+1) + j)*(n+1) + i and coordinates
    (x_i, x_j, x_k).  Cell tets follow the 6 monotone lattice paths from the
    cell's v000 corner to its v111 corner, one per axis permutation.  Returned
    tets are NOT re-oriented (half of them are negatively oriented), which the
    consumers must handle.

    Returns (vertices float64 [nv,3], tets int32 [nt,4]).
    """
    m = n + 1
    x = grid_coords(n)
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    verts = np.stack([x[ii.ravel()], x[jj.ravel()], x[kk.ravel()]], axis=1)

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()

    def vid(di, dj, dk):
        return ((ck + dk) * m + (cj + dj)) * m + (ci + di)

    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for p in perms:
        cur = [0, 0, 0]
        path = [vid(*cur)]
        for ax in p:
            cur[ax] += 1
            path.append(vid(*cur))
        tets.append(np.stack(path, axis=1))
    # interleave so the 6 tets of a cell are consecutive
    t = np.stack(tets, axis=1).reshape(-1, 4)
    return verts, t.astype(np.int32)


def interior_vertex_mask(n: int) -> np.ndarray:
    m = n + 1
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    inside = lambda a: (a > 0) & (a < n)
    return (inside(ii) & inside(jj) & inside(kk)).ravel()


def signed_volumes6(verts: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """6 x signed volume of each tet (input validation only)."""
    a, b, c, d = (verts[tets[:, k]] for k in range(4))
    return np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a))


def jitter_interior(verts: np.ndarray, tets: np.ndarray, n: int, rng: np.random.Generator,
                    frac: float = 0.2, max_redraws: int = 1000) -> np.ndarray:
    """Move every interior vertex by U[-frac*h, frac*h]^3 (h = 2/n).

    All displacements are drawn at once in vertex-index order; any vertex that
    leaves an incident tet with non-positive volume (relative to the tet's
    original orientation) is redrawn, in vertex-index order, until none does.
    """
    h = 2.0 / n
    out = verts.copy()
    mask = interior_vertex_mask(n)
    idx = np.nonzero(mask)[0]
    out[idx] += rng.uniform(-frac * h, frac * h, size=(idx.size, 3))
    sign0 = np.sign(signed_volumes6(verts, tets))
    for _ in range(max_redraws):
        bad = np.nonzero(signed_volumes6(out, tets) * sign0 <= 0)[0]
        if bad.size == 0:
            return out
        bad_v = np.unique(tets[bad].ravel())
        bad_v = bad_v[mask[bad_v]]
        for v in bad_v:
            out[v] = verts[v] + rng.uniform(-frac * h, frac * h, size=3)
    raise RuntimeError("jitter_interior: could not produce a valid mesh")


def cubic_map(verts: np.ndarray) -> np.ndarray:
    """x -> sign(x)|x|^3 per axis (maps [-1,1]^3 onto itself)."""
    return np.sign(verts) * np.abs(verts) ** 3


def tet_centroids(verts: np.ndarray, tets: np.ndarray) -> np.ndarray:
    return verts[tets].mean(axis=1)


def phantom_params(rng: np.random.Generator):
    """Three axis-aligned ellipsoids: centres U[-0.4,0.4]^3, semi-axes U[0.2,0.6]^3."""
    centres = rng.uniform(-0.4, 0.4, size=(3, 3))
    axes = rng.uniform(0.2, 0.6, size=(3, 3))
    values = np.array([0.2, 0.5, 1.0])
    return centres, axes, values


def phantom_at(points: np.ndarray, centres, axes, values) -> np.ndarray:
    """Sum of the ellipsoid indicator values at each point (overlaps add)."""
    out = np.zeros(points.shape[0])
    for c, a, v in zip(centres, axes, values):
        r2 = (((points - c) / a) ** 2).sum(axis=1)
        out += np.where(r2 <= 1.0, v, 0.0)
    return out


# --------------------------------------------------------------------------
# cone-beam geometry (parameters only; ray construction lives with each consumer)
# --------------------------------------------------------------------------

@dataclass
class ConeBeam:
    """Circular cone-beam scan: source at ``dso`` from the z axis, flat detector
    at ``dsd`` from the source, ``nu`` x ``nv`` pixels of pitch (du, dv),
    angles in radians.  Projections are laid out proj[angle][iv][iu][c]."""
    dso: float
    dsd: float
    nu: int
    nv: int
    du: float
    dv: float
    angles: np.ndarray

    @property
    def nangles(self) -> int:
        return int(self.angles.size)

    @property
    def nrays(self) -> int:
        return self.nangles * self.nu * self.nv


def uniform_angles(n: int) -> np.ndarray:
    """theta_a = 2*pi*a/n, a = 0..n-1 (endpoint excluded)."""
    return 2.0 * np.pi * np.arange(n, dtype=np.float64) / n


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n_cells: int
    verts: np.ndarray
    tets: np.ndarray
    mu: np.ndarray          # [nt] or [nt, C]
    geom: ConeBeam
    channels: int = 1
    extra: dict = field(default_factory=dict)


def config1(n_cells: int = 8, det: int = 64, pitch: float = 0.1, nangles: int = 32) -> Workload:
    """Plain method, tiny: Kuhn 8^3 (3072 tets), mu ~ U[0,1], 64x64 det, 32 angles."""
    rng = rng_for(0)
    verts, tets = kuhn_cube(n_cells)
    mu = rng.uniform(0.0, 1.0, size=tets.shape[0])
    g = ConeBeam(4.0, 8.0, det, det, pitch, pitch, uniform_angles(nangles))
    return Workload("kuhn8_det64x64_a32", n_cells, verts, tets, mu, g)


def config2(n_cells: int = 96, det: int = 512, pitch: float = 0.0125, nangles: int = 360) -> Workload:
    """Plain method at scale: jittered Kuhn 96^3 (5.3M tets), phantom + N(0, 0.01)."""
    rng = rng_for(1)
    verts, tets = kuhn_cube(n_cells)
    verts = jitter_interior(verts, tets, n_cells, rng)
    centres, axes, values = phantom_params(rng)
    mu = phantom_at(tet_centroids(verts, tets), centres, axes, values)
    mu = mu + rng.normal(0.0, 0.01, size=mu.size)
    g = ConeBeam(4.0, 8.0, det, det, pitch, pitch, uniform_angles(nangles))
    return Workload(f"jittered_kuhn{n_cells}_det{det}x{det}_a{nangles}", n_cells, verts, tets,
                    mu.astype(np.float32).astype(np.float64), g)


def config3(n_cells: int = 64, det: int = 256, pitch: float = 0.025, nangles: int = 180,
            n_adversarial: int = 1_000_000) -> Workload:
    """Robustness: cubic-mapped Kuhn 64^3 and adversarial rays aimed exactly at
    vertices, edge midpoints and points of interior faces."""
    rng = rng_for(2)
    verts, tets = kuhn_cube(n_cells)
    verts = cubic_map(verts)
    mu = rng.uniform(0.0, 1.0, size=tets.shape[0])
    g = ConeBeam(4.0, 8.0, det, det, pitch, pitch, uniform_angles(nangles))
    w = Workload(f"cubic_kuhn{n_cells}_det{det}x{det}_a{nangles}", n_cells, verts, tets, mu, g)
    if n_adversarial:
        S, T, kind = adversarial_rays(verts, tets, n_cells, n_adversarial, rng_for(2, 1))
        w.extra.update(adv_src=S, adv_target=T, adv_kind=kind)
    return w


def config4(n_cells: int = 64, det: int = 256, pitch: float = 0.025, nangles: int = 180) -> Workload:
    """Differentiation: jittered Kuhn 64^3, ground truth = phantom (no noise)."""
    rng = rng_for(3)
    verts, tets = kuhn_cube(n_cells)
    verts = jitter_interior(verts, tets, n_cells, rng)
    centres, axes, values = phantom_params(rng)
    mu_true = phantom_at(tet_centroids(verts, tets), centres, axes, values)
    g = ConeBeam(4.0, 8.0, det, det, pitch, pitch, uniform_angles(nangles))
    w = Workload(f"recon_kuhn{n_cells}_det{det}x{det}_a{nangles}", n_cells, verts, tets, mu_true, g)
    w.extra["noise_rng"] = rng_for(3, 1)
    return w


def config5_specs(n_problems: int = 24, seed_stream: int = 0):
    """Per-problem sizes for the batched workload: cells/side log-uniform in
    [16, 128), detector side log-uniform in [128, 1024] (pitch 6.4/N), angle
    count log-uniform in [60, 720]."""
    rng = rng_for(4, seed_stream)
    specs = []
    for _ in range(n_problems):
        n = int(round(math.exp(rng.uniform(math.log(16), math.log(128)))))
        N = int(round(math.exp(rng.uniform(math.log(128), math.log(1024)))))
        na = int(round(math.exp(rng.uniform(math.log(60), math.log(720)))))
        specs.append((n, N, na))
    return specs


def config5_problem(k: int, n: int, N: int, na: int, channels: int = 4) -> Workload:
    """Problem k of the batched workload: jittered Kuhn n^3, C-channel mu ~ U[0,1]."""
    rng = rng_for(4, 100 + k)
    verts, tets = kuhn_cube(n)
    verts = jitter_interior(verts, tets, n, rng)
    mu = rng.uniform(0.0, 1.0, size=(tets.shape[0], channels)).astype(np.float32).astype(np.float64)
    pitch = 6.4 / N
    g = ConeBeam(4.0, 8.0, N, N, pitch, pitch, uniform_angles(na))
    return Workload(f"batch{k}_kuhn{n}_det{N}_a{na}", n, verts, tets, mu, g, channels=channels)


# --------------------------------------------------------------------------
# explicit rays
# --------------------------------------------------------------------------

def unique_edges(tets: np.ndarray) -> np.ndarray:
    pairs = np.concatenate([tets[:, [i, j]] for i in range(4) for j in range(i + 1, 4)])
    pairs.sort(axis=1)
    return np.unique(pairs, axis=0)


def boundary_vertex_mask(verts: np.ndarray) -> np.ndarray:
    return (np.abs(verts) == 1.0).any(axis=1)


def adversarial_rays(verts, tets, n_cells, count, rng):
    """Rays from random points of the radius-4, z=0 source circle aimed exactly at
    (1/3 each) interior vertices, midpoints (a+b)*0.5 of uniformly chosen
    edges, and uniform points of uniformly chosen interior faces.

    Returns (sources [count,3], targets [count,3], kind [count] in {0,1,2}).
    """
    k0 = count // 3
    k1 = count // 3
    k2 = count - k0 - k1
    phi = rng.uniform(0.0, 2.0 * np.pi, size=count)
    src = np.stack([4.0 * np.cos(phi), 4.0 * np.sin(phi), np.zeros(count)], axis=1)

    interior = np.nonzero(~boundary_vertex_mask(verts))[0]
    tv = verts[interior[rng.integers(0, interior.size, size=k0)]]

    edges = unique_edges(tets)
    e = edges[rng.integers(0, edges.shape[0], size=k1)]
    tm = (verts[e[:, 0]] + verts[e[:, 1]]) * 0.5

    # interior faces: (tet, local face) pairs whose 3 vertices are not all on one
    # cube face; each interior face appears twice among all pairs, so uniform
    # rejection sampling over pairs is uniform over interior faces.
    on_plane = np.abs(verts) == 1.0
    pts = []
    need = k2
    while need > 0:
        t = rng.integers(0, tets.shape[0], size=2 * need)
        f = rng.integers(0, 4, size=2 * need)
        tri = np.stack([tets[t, (f + 1) % 4], tets[t, (f + 2) % 4], tets[t, (f + 3) % 4]], axis=1)
        bnd = (on_plane[tri[:, 0]] & on_plane[tri[:, 1]] & on_plane[tri[:, 2]]).any(axis=1)
        tri = tri[~bnd][:need]
        w = rng.dirichlet([1.0, 1.0, 1.0], size=tri.shape[0])
        pts.append(np.einsum("ij,ijk->ik", w, verts[tri]))
        need -= tri.shape[0]
    tf = np.concatenate(pts)
    targets = np.concatenate([tv, tm, tf])
    kind = np.concatenate([np.zeros(k0, np.int8), np.ones(k1, np.int8), np.full(k2, 2, np.int8)])
    return src, targets, kind


def random_rays_through_box(count: int, rng: np.random.Generator, radius: float = 4.0):
    """Generic rays: sources on a sphere of the given radius, aimed at uniform
    points of [-1.2, 1.2]^3 (some miss the cube)."""
    v = rng.normal(size=(count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    src = radius * v
    tgt = rng.uniform(-1.2, 1.2, size=(count, 3))
    return src, tgt
