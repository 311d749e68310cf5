"""rb_gepp_solve_static: the batched partial-pivot solve that allocates nothing.

Callers that cannot allocate device memory while they solve (under a fixed memory budget, with
only lent buffers, or on a hot path that must not take the allocator's locks) use this entry
point; its working matrices live
in a file-scope device array that every call shares. The test calls it through the C ABI on
caller-owned device buffers, several times in a row with different sizes (the shared array
keeps the previous call's contents), and compares each result with the allocating entry point
rb_gepp_solve and with the oracle's elimination. The cases include batches larger than the
grid, so that one CTA solves several systems in turn through the same slice of the array, a
singular system among a CTA's later systems, and the largest accepted size.
This file is collected last so that a run stopping at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def static_grid(rb, n, batch, sms):
    """The grid the entry point launches: one system per CTA at a time, as many CTAs as the
    array holds systems of size n, at most 8 per SM and at most the batch."""
    per = n * n * 8
    return min(rb.RB_STATIC_SCRATCH_BYTES // per, 8 * sms, batch)


# (n, batch, singular systems): ragged batches; batches beyond the grid (n = 300: 23 CTAs for
# 64 systems; n = 512 = RB_STATIC_N_MAX: 8 CTAs for 20 systems), each with a singular system
# that its CTA reaches after solving others
CASES = [(37, 300, (5,)), (64, 129, (0, 128)), (300, 64, (50,)), (512, 20, (17,))]


def test_static_solve_matches_allocating_solve_and_oracle(rb):
    import torch
    g = np.random.default_rng(20240611)
    stream = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for n, batch, singular in CASES:  # one call after another; the array is reused
        M = g.standard_normal((batch, n, n))
        for s in singular:
            M[s] = 0.0
            M[s, : n // 2] = g.standard_normal((n // 2, n))  # rank-deficient, not all zero
        rhs = g.standard_normal((batch, n))
        if n > 64:
            assert static_grid(rb, n, batch, sms) < batch  # CTAs reuse their slice
        with rb.Context() as ctx:
            x_ref, st_ref = ctx.rb_gepp_solve(M, rhs)
        x_or, st_or = oracle.gepp_solve(M, rhs)
        dM = torch.from_numpy(M).cuda()
        drhs = torch.from_numpy(rhs).cuda()
        dx = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
        dst = torch.full((batch,), -7, dtype=torch.int32, device="cuda")
        rc = rb.rb_gepp_solve_static(n, batch, dM, drhs, dx, dst, stream)
        torch.cuda.synchronize()
        assert rc == rb.RB_OK, rb.rb_last_error_global()
        st = dst.cpu().numpy()
        x = dx.cpu().numpy()
        expect_sing = np.zeros(batch, bool)
        expect_sing[list(singular)] = True
        np.testing.assert_array_equal(st != 0, expect_sing)
        np.testing.assert_array_equal(st, st_ref)
        np.testing.assert_array_equal(st, st_or)
        ok = st == 0
        # the same elimination as the allocating entry point
        np.testing.assert_allclose(x[ok], x_ref[ok], rtol=1e-12, atol=1e-14)
        # the oracle: the same pivots, another rounding order; backward-stable GEPP bounds the
        # difference by a small multiple of n eps cond(M)
        cond = np.linalg.cond(M[ok])
        err = np.linalg.norm(x[ok] - x_or[ok], axis=1) / np.linalg.norm(x_or[ok], axis=1)
        assert np.all(err <= 10 * n * np.finfo(float).eps * cond), (n, err.max())
        # the inputs are not modified
        np.testing.assert_array_equal(dM.cpu().numpy(), M)
        np.testing.assert_array_equal(drhs.cpu().numpy(), rhs)


def test_static_solve_rejects_oversize(rb):
    import torch
    n = rb.RB_STATIC_N_MAX + 1
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = rb.rb_gepp_solve_static(n, 1, d, d, d, s, None)
    assert rc == rb.RB_ERR_ARG
    assert str(rb.RB_STATIC_N_MAX) in rb.rb_last_error_global()
    assert rb.rb_gepp_solve_static(0, 1, d, d, d, s, None) == rb.RB_ERR_ARG
