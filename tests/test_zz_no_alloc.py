"""rb_gepp_solve_static: the batched partial-pivot solve that allocates nothing.

Callers that cannot allocate device memory while they solve (inside a graph capture, under a
fixed memory budget, or with only lent buffers) use this entry point; its working matrices live
in a file-scope device array. The test calls it through the C ABI on caller-owned device
buffers, twice in a row with different sizes (the shared array keeps the previous call's
contents), and compares with the allocating rb_gepp_solve, which runs the same elimination.
This file is collected last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def test_static_solve_matches_allocating_solve(rb):
    import torch
    g = np.random.default_rng(20240611)
    stream = torch.cuda.current_stream().cuda_stream
    for n, batch in ((37, 300), (64, 129)):  # two calls in a row; ragged batch sizes
        M = g.standard_normal((batch, n, n))
        M[5] = 0.0  # one singular system
        rhs = g.standard_normal((batch, n))
        with rb.Context() as ctx:
            x_ref, st_ref = ctx.rb_gepp_solve(M, rhs)
        dM = torch.from_numpy(M).cuda()
        drhs = torch.from_numpy(rhs).cuda()
        dx = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
        dst = torch.full((batch,), -7, dtype=torch.int32, device="cuda")
        rc = rb.rb_gepp_solve_static(n, batch, dM, drhs, dx, dst, stream)
        torch.cuda.synchronize()
        assert rc == rb.RB_OK, rb.rb_last_error_global()
        st = dst.cpu().numpy()
        x = dx.cpu().numpy()
        np.testing.assert_array_equal(st, st_ref)
        ok = st == 0
        np.testing.assert_allclose(x[ok], x_ref[ok], rtol=1e-12, atol=1e-14)
        # the inputs are not modified
        np.testing.assert_array_equal(dM.cpu().numpy(), M)


def test_static_solve_rejects_oversize(rb):
    import torch
    n = rb.RB_STATIC_N_MAX + 1
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = rb.rb_gepp_solve_static(n, 1, d, d, d, s, None)
    assert rc == rb.RB_ERR_ARG
    assert str(rb.RB_STATIC_N_MAX) in rb.rb_last_error_global()
