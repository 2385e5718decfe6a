"""The multi-GPU angle split (Sec. II-F) on the CPU: gloo ranks, world size 2
and 3, the oracle standing in for each rank's projector.

Each rank takes its block of angles (split.angle_range), backprojects y over
those angles only (oracle.backward_cone on the sub-scan), and split.
allreduce_sum adds the ranks' per-tet buffers.  The result must equal the
oracle's backprojection of the whole scan (Eq. 3: x_i = sum_j a_ij y_j over
all rays j), and each rank's forward projection must equal its rows of the
whole scan's (Eq. 2; rays are independent, no exchange).  No GPU: the same
functions run over NCCL between GPUs with the library's kernels."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_angle_range_partitions():
    from paper_1908_06909_gb300.split import angle_range
    for n in (0, 1, 5, 32, 360, 361):
        for world in (1, 2, 3, 4, 8):
            blocks = [angle_range(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(ValueError):
        angle_range(10, 2, 2)


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    from paper_1908_06909_gb300.split import allreduce_sum, angle_range
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.config1(n_cells=4, det=12, pitch=0.5, nangles=7)
    g = w.geom
    rng = np.random.default_rng(5)
    shape = (g.nangles, g.nv, g.nu)
    y = rng.uniform(0.0, 1.0, size=shape)            # the whole scan's data, same on every rank
    a0, a1 = angle_range(g.nangles, rank, world)
    sub = W.ConeBeam(g.dso, g.dsd, g.nu, g.nv, g.du, g.dv, g.angles[a0:a1])
    x_local = oracle.backward_cone(w.verts, w.tets, y[a0:a1].reshape(-1), sub)
    x = allreduce_sum(torch.tensor(x_local))
    p_local = oracle.forward_cone(w.verts, w.tets, w.mu, sub)
    out.put((rank, a0, a1, x.numpy(), p_local))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_angle_split_backprojection_sums_to_whole_scan(world):
    import sys
    sys.path.insert(0, ROOT)
    import torch.multiprocessing as mp
    import oracle
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    import queue
    import time
    got, t0 = [], time.time()
    while len(got) < world:  # fail fast if a rank dies instead of waiting out a timeout
        try:
            got.append(q.get(timeout=2))
        except queue.Empty:
            assert all(p.exitcode in (None, 0) for p in procs), [p.exitcode for p in procs]
            assert time.time() - t0 < 300, "ranks did not report"
    res = sorted(got, key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = W.config1(n_cells=4, det=12, pitch=0.5, nangles=7)
    rng = np.random.default_rng(5)
    shape = (w.geom.nangles, w.geom.nv, w.geom.nu)
    y = rng.uniform(0.0, 1.0, size=shape)
    want = oracle.backward_cone(w.verts, w.tets, y.reshape(-1), w.geom)
    whole = oracle.forward_cone(w.verts, w.tets, w.mu, w.geom).reshape(shape)
    assert [r[1] for r in res] == sorted(r[1] for r in res) and res[-1][2] == w.geom.nangles
    for rank, a0, a1, x, p_local in res:
        assert np.allclose(x, want, rtol=1e-12, atol=1e-14)          # every rank holds A^T y
        assert np.array_equal(p_local.reshape(a1 - a0, *shape[1:]), whole[a0:a1])
    assert want.max() > 0
