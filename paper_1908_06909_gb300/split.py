"""Projections split across GPUs by angle (Sec. II-F, multi-GPU paragraph).

The paper spreads the projection angles of one scan over several GPUs, each
holding the whole mesh.  Rays are independent, so the forward projection of
an angle needs nothing from another GPU; the backprojection of the whole scan,
x = A^T y = sum over angle ranges of A_r^T y_r, needs one sum of the per-tet
buffers across GPUs.  Here one process drives one GPU (torch.distributed,
NCCL between GPUs): rank r owns the contiguous angle range angle_range(N, r, R)
and its own replica of the mesh, projects only its angles, and the
backprojection adds the ranks' partial per-tet sums with a single all-reduce.

Everything here is host logic around the library's kernels and one
collective; the same functions run over gloo on the CPU in the tests, with the
oracle standing in for the per-rank projector.
"""
from __future__ import annotations


def angle_range(nangles: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block [a0, a1) of the angles owned by `rank`: the first
    nangles % world ranks get one angle more than the others, so block sizes
    differ by at most one and the blocks tile 0..nangles-1 in rank order."""
    if world < 1 or not 0 <= rank < world or nangles < 0:
        raise ValueError("need 0 <= rank < world and nangles >= 0")
    q, r = divmod(nangles, world)
    a0 = rank * q + min(rank, r)
    return a0, a0 + q + (1 if rank < r else 0)


def allreduce_sum(x, group=None):
    """x <- the sum of x over the ranks of `group` (in place; returns x).  With
    no process group (a single process) x is returned unchanged."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


class AngleSplit:
    """One rank's share of a scan: its block of angles, projected with the
    library's kernels against its replica of the mesh.

    mesh: this rank's tp.Mesh (on its GPU); cone: an object with dso, dsd, nu,
    nv, du, dv and the full angle list; rank / world default to the process
    group's.  forward(mu) returns this rank's projections [a1 - a0, nv, nu(,C)];
    backward(y_local) returns the full x = A^T y on every rank (the local
    backprojection, then the all-reduce)."""

    def __init__(self, mesh, cone, rank=None, world=None, group=None, options=None):
        import numpy as np
        import torch.distributed as dist
        from . import Geometry
        if rank is None or world is None:
            if dist.is_available() and dist.is_initialized():
                rank, world = dist.get_rank(group), dist.get_world_size(group)
            else:
                rank, world = 0, 1
        self.rank, self.world, self.group = rank, world, group
        angles = np.asarray(cone.angles, dtype=np.float64)
        self.a0, self.a1 = angle_range(angles.size, rank, world)
        self.mesh, self.options = mesh, options
        self.geo = Geometry(cone.dso, cone.dsd, cone.nu, cone.nv, cone.du, cone.dv,
                            angles[self.a0:self.a1]) if self.a1 > self.a0 else None

    def forward(self, mu, out=None):
        from . import forward
        if self.geo is None:
            return None
        return forward(self.mesh, self.geo, mu, out=out, options=self.options)

    def backward(self, y_local, out=None):
        import torch
        from . import backward
        if self.geo is None:
            ext = tuple(y_local.shape[3:]) if y_local is not None and y_local.dim() == 4 else ()
            dtype = torch.float32 if y_local is None else y_local.dtype
            x = torch.zeros((self.mesh.nt,) + ext, dtype=dtype, device="cuda")
        else:
            x = backward(self.mesh, self.geo, y_local, out=out, options=self.options)
        return allreduce_sum(x, self.group)
