"""tetproj_backward_noalloc against tetproj_backward (GPU).

Some callers cannot call cudaMalloc when they backproject (their device memory
is owned by another allocator, or they must not pay cudaMalloc's implicit
synchronisation), so the library offers a backprojection whose scratch is a
fixed device array inside the library.  This test calls it through the C ABI,
twice in a row (the array keeps the previous call's contents, so the second
call checks that everything that must start at zero is cleared), and compares
each result with tetproj_backward within the parity tolerance of the GPU tests:
per tet |x_noalloc - x_backward| <= tau * sum_j a_ij |y_j| (tau = 1e-12 plain
FP64, 1e-5 filtered FP32).  It runs alone or after the other tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_backward_noalloc_matches_backward(prec):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1908_06909_gb300 as tp
    dt = torch.float64 if prec == "f64" else torch.float32
    tau = 1e-12 if prec == "f64" else 1e-5
    w = W.config1()
    mesh = tp.Mesh(w.verts, w.tets)
    geo = tp.Geometry.from_cone(w.geom)
    gen = torch.Generator("cuda").manual_seed(17)
    for call in range(2):
        y = torch.rand(geo.shape, dtype=dt, device="cuda", generator=gen)
        if call == 1:
            y = y * 3.0 - 1.0  # different values and signs on the second call
        ref = tp.backward(mesh, geo, y)
        mag = tp.backward(mesh, geo, y.abs())
        out = tp.backward_noalloc(mesh, geo, y)
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).abs()
        bound = tau * mag.double() + 1e-300
        assert bool((err <= bound).all()), (call, float((err / bound).max()))
        assert float(mag.max()) > 0
    st = mesh.stats()
    assert st["error"] == 0
