"""The angle split (Sec. II-F) through the library's kernels, one process:
the ranks' shares are computed one after another on the same GPU (no
process group, so no collective and no rank waits for another), and their
sum must equal the whole scan's backprojection; each rank's forward equals
its block of the whole scan's projection.  The cross-rank sum itself is
tested over gloo in test_angle_split.py."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [1, 3, 8])
def test_angle_split_shares_sum_to_whole_scan(world):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    from paper_1908_06909_gb300.split import AngleSplit
    w = W.config1(nangles=20)
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    mu = torch.tensor(w.mu, dtype=torch.float64, device="cuda")
    o = tp.make_options(precision=tp.PLAIN_FP64)
    whole = tp.forward(mesh, geo, mu, options=o)
    y = torch.rand(geo.shape, dtype=torch.float64, device="cuda",
                   generator=torch.Generator("cuda").manual_seed(3))
    want = tp.backward(mesh, geo, y, options=o)
    mag = tp.backward(mesh, geo, y.abs(), options=o)
    total = torch.zeros_like(want)
    for r in range(world):
        s = AngleSplit(mesh, w.geom, rank=r, world=world, options=o)
        if s.geo is None:
            continue
        assert torch.equal(s.forward(mu), whole[s.a0:s.a1])
        total += s.backward(y[s.a0:s.a1].contiguous())  # no process group: the local share
    torch.cuda.synchronize()
    assert bool(((total - want).abs() <= 1e-12 * mag + 1e-300).all())
