"""Robustness of the mixed path on the GPU: the inexact Newton on a weakly damped problem (the
viscous terms weakened 64 times, several iterations far from the root), and a device-side wait
of the tensor-core pipeline that runs out (bounded waits, error status, a usable context
afterwards)."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


@pytest.mark.parametrize("n,damp", [(30, 64.0), (48, 64.0), (40, 256.0)])
def test_weakly_damped_mixed(rb, n, damp, monkeypatch):
    """A/64 (A/256) leaves the small-data regime the workloads are scaled into: the first Newton
    steps are far from the root and the inexact Jacobian's chord steps contract slowly. Every
    query must either match the oracle within the mixed tolerance or report that it did not
    converge (never a wrong answer with status OK); where the oracle converges, the mixed path
    must too."""
    monkeypatch.setenv("RB_SMALL", "0")  # the tensor-core pipeline's inexact Newton
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n)
    ops.A = ops.A / damp
    q = synth.make_queries(wl, batch=250, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, inf_ref = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    ok = info["status"] == rb.RB_Q_OK
    assert set(np.unique(info["status"])) <= {rb.RB_Q_OK, rb.RB_Q_NOT_CONVERGED, rb.RB_Q_NONFINITE}
    both = ok & (inf_ref["status"] == 0)
    assert rel(u[both], u_ref[both]).max() <= TOL_MIXED
    assert rel(p[both], p_ref[both]).max() <= 10 * TOL_MIXED
    # the mixed path converges wherever the oracle does: a query whose chord steps stall asks
    # for a fresh Jacobian, and one that stalls with it too is solved by the FP64 Newton
    # (reported as precision_used = RB_PREC_FP64)
    assert np.all(ok[inf_ref["status"] == 0]), (np.sum(~ok), info["iters"].max())
    assert set(np.unique(info["precision_used"])) <= {rb.RB_PREC_MIXED, rb.RB_PREC_FP64}
    # more iterations than the damped workloads (3-4): the problem is harder, not broken
    assert info["iters"][both].max() >= 5
    if damp >= 256:
        assert np.any(info["precision_used"] == rb.RB_PREC_FP64)


@pytest.mark.parametrize("graph", [0, 1])
def test_bounded_wait_runs_out(rb, monkeypatch, graph):
    """One stage of the single-CTA Jacobian GEMM waits for 16 bytes that never arrive
    (RB_TEST_WAIT_DEFICIT=1): its consumer's wait gives up after its time limit, every role of
    the kernel leaves, and the solve reports RB_ERR_TIMEOUT. The same context then solves
    correctly, and so does a fresh one."""
    monkeypatch.setenv("RB_GEMM_PAIRS", "0")  # single CTAs: no cluster barriers involved
    monkeypatch.setenv("RB_SMALL", "0")  # the tensor-core pipeline also at n = 16
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=16)
    q = synth.make_queries(wl, batch=8, n_max=16)
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(q.mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED, use_graph=graph, autotune=0) as ctx:
        ctx.load_set(ops)
        monkeypatch.setenv("RB_TEST_WAIT_DEFICIT", "1")
        t0 = time.perf_counter()
        with pytest.raises(rb.RbError) as ei:
            ctx.rb_solve(q.mu)
        dt = time.perf_counter() - t0
        assert ei.value.code == rb.RB_ERR_TIMEOUT, str(ei.value)
        assert dt < 30.0, dt
        monkeypatch.delenv("RB_TEST_WAIT_DEFICIT")
        # another batch shape, so that the graph path captures a new graph without the deficit
        u, p, info = ctx.rb_solve(q.mu[:7])
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref[:7]).max() <= TOL_MIXED and rel(p, p_ref[:7]).max() <= 10 * TOL_MIXED
    with rb.Context(rb.RB_PREC_MIXED, use_graph=graph, autotune=0) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(q.mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL_MIXED
