"""Continuous-batching server (rb_serve_*): results are the same alone and in the mix, agree with
rb_solve and the oracle, admission waits for memory, and cancellation completes every ticket."""
import threading
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


def wait(ctx, ticket, timeout=60.0):
    t0 = time.time()
    while True:
        r = ctx.rb_serve_poll(ticket)
        if r is not None:
            return r
        if time.time() - t0 > timeout:
            raise TimeoutError(ticket)
        time.sleep(1e-4)


@pytest.fixture(scope="module")
def sweep():
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=40)
    q = synth.make_queries(wl, batch=600, n_max=40)
    return wl, ops, q


def test_alone_equals_in_the_mix(rb, sweep):
    wl, ops, q = sweep
    probe = np.array([17.5, 420.0])
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        ctx.rb_serve_start()
        u1, p1, i1 = wait(ctx, ctx.rb_serve_submit(probe))
        # a stream of arrivals from another thread while the probe is resubmitted mid-stream
        tickets = []

        def feeder():
            for k in range(len(q.mu)):
                tickets.append(ctx.rb_serve_submit(q.mu[k]))
                if k % 50 == 0:
                    time.sleep(2e-4)

        th = threading.Thread(target=feeder)
        th.start()
        time.sleep(1e-3)
        tp = ctx.rb_serve_submit(probe)
        th.join()
        u2, p2, i2 = wait(ctx, tp)
        res = [wait(ctx, t) for t in tickets]
        p50, p99, sps = ctx.rb_serve_stats()
        ctx.rb_serve_stop(True)
        U = np.stack([r[0] for r in res])
        P = np.stack([r[1] for r in res])
        st = np.array([r[2]["status"] for r in res])
        u_ref, p_ref, info_ref = ctx.rb_solve(q.mu)
    assert i1["status"] == 0 and i2["status"] == 0
    assert rel(u2, u1) <= TOL_MIXED and rel(p2, p1) <= 10 * TOL_MIXED
    assert np.all(st == 0)
    assert rel(U, u_ref).max() <= TOL_MIXED
    assert rel(P, p_ref).max() <= 10 * TOL_MIXED
    o = oracle.Oracle.from_set(ops)
    idx = np.arange(0, len(q.mu), 37)
    u_or, p_or, _ = o.solve(q.mu[idx], threads=8)
    assert rel(U[idx], u_or).max() <= TOL_MIXED
    assert 0 < p50 <= p99 and sps > 0


def test_admission_waits_for_slots(rb, sweep):
    wl, ops, q = sweep
    # 8 device slots for 200 queries: later queries wait until earlier ones free their slots
    with rb.Context(rb.RB_PREC_MIXED, serve_slots=8) as ctx:
        ctx.load_set(ops)
        ctx.rb_serve_start()
        assert ctx.rb_serve_slots() == 8
        tickets = [ctx.rb_serve_submit(q.mu[k]) for k in range(200)]
        res = [wait(ctx, t) for t in tickets]
        ctx.rb_serve_stop(True)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u_ref, _, _ = ctx.rb_solve(q.mu[:200])
    U = np.stack([r[0] for r in res])
    assert all(r[2]["status"] == 0 for r in res)
    assert rel(U, u_ref).max() <= TOL_MIXED


def test_budget_too_small_for_any_slot(rb, sweep):
    wl, ops, q = sweep
    with rb.Context(rb.RB_PREC_MIXED, mem_budget=12 << 20) as ctx:
        try:
            ctx.load_set(ops)
        except rb.RbError:
            pytest.skip("operators alone exceed this budget")
        with pytest.raises(rb.RbError) as ei:
            ctx.rb_serve_start()
        assert ei.value.code == rb.RB_ERR_OOM


def test_cancel_and_argument_errors(rb, sweep):
    wl, ops, q = sweep
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        with pytest.raises(rb.RbError):
            ctx.rb_serve_submit(q.mu[0])  # not started
        ctx.rb_serve_start()
        with pytest.raises(rb.RbError):
            ctx.rb_serve_submit(q.mu[0], n=41)  # n out of range
        with pytest.raises(rb.RbError):
            ctx.rb_solve(q.mu[:2])  # the server owns the batch state
        tickets = [ctx.rb_serve_submit(q.mu[k]) for k in range(400)]
        ctx.rb_serve_stop(False)  # cancel
        res = [wait(ctx, t) for t in tickets]
        st = np.array([r[2]["status"] for r in res])
        assert set(np.unique(st)) <= {rb.RB_Q_OK, rb.RB_Q_REJECTED}
        with pytest.raises(rb.RbError):
            ctx.rb_serve_poll(tickets[0])  # released after the first successful poll
        with pytest.raises(rb.RbError):
            ctx.rb_serve_submit(q.mu[0])  # stopped


def test_fp64_server_and_sizes(rb, sweep):
    wl, ops, q = sweep
    sizes = [40, 7, 33, 1, 20]
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        ctx.rb_serve_start()
        tickets = [ctx.rb_serve_submit(q.mu[k], n=sizes[k % 5]) for k in range(50)]
        res = [wait(ctx, t) for t in tickets]
        ctx.rb_serve_stop(True)
    o = oracle.Oracle.from_set(ops)
    n = np.array([sizes[k % 5] for k in range(50)], dtype=np.int32)
    u_or, _, _ = o.solve(q.mu[:50], n=n, threads=8)
    U = np.stack([r[0] for r in res])
    assert all(r[2]["status"] == 0 for r in res)
    assert rel(U, u_or).max() <= 1e-10


def test_mixed_server_sizes_in_buckets(rb):
    """Mixed-precision serving of queries of different sizes: every step runs each size bucket's
    slots as one batch (gathered, iterated, scattered back); velocity and pressure match the
    oracle per size, and a query gives the same result alone and among the others."""
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=72)
    q = synth.make_queries(wl, batch=240, n_max=72)
    sizes = [72, 9, 33, 50, 64, 17, 1, 70]
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        ctx.rb_serve_start()
        alone = wait(ctx, ctx.rb_serve_submit(q.mu[5], n=sizes[5]))
        tickets = [ctx.rb_serve_submit(q.mu[k], n=sizes[k % len(sizes)]) for k in range(len(q.mu))]
        res = [wait(ctx, t) for t in tickets]
        ctx.rb_serve_stop(True)
    n = np.array([sizes[k % len(sizes)] for k in range(len(q.mu))], dtype=np.int32)
    o = oracle.Oracle.from_set(ops)
    u_or, p_or, _ = o.solve(q.mu, n=n, threads=8)
    U = np.stack([r[0] for r in res])
    P = np.stack([r[1] for r in res])
    assert all(r[2]["status"] == 0 for r in res)
    for s in sizes:
        k = n == s
        assert rel(U[k][:, :s], u_or[k][:, :s]).max() <= TOL_MIXED, s
        assert np.all(U[k][:, s:] == 0)
    assert rel(P, p_or).max() <= 10 * TOL_MIXED
    assert rel(res[5][0], alone[0]) <= TOL_MIXED and rel(res[5][1], alone[1]) <= 10 * TOL_MIXED


@pytest.mark.timeout(900)
def test_serve_n160_shape_batch_and_server(rb):
    """The serving workload's own shape (n_max = 160, Q_a = Q_c = 16, Q_f = 4, C FP32-exact): 72
    queries with sizes spread over [16, 160] (both ends included) and parameters over the box
    (corners included), solved as one batch and through the server, both against the oracle."""
    wl = synth.WORKLOADS["serve_n160"]
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl, batch=68)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    sizes = np.linspace(16, 160, len(mu)).round().astype(np.int32)
    sizes = np.random.default_rng(7).permutation(sizes)
    assert sizes.min() == 16 and sizes.max() == 160
    o = oracle.Oracle.from_set(ops)
    u_or, _, inf_or = o.solve(mu, n=sizes, threads=oracle.max_threads())
    assert np.all(inf_or["status"] == 0)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u_b, _, info_b = ctx.rb_solve(mu, n=sizes)
        ctx.rb_serve_start()
        tickets = [ctx.rb_serve_submit(mu[k], n=int(sizes[k])) for k in range(len(mu))]
        res = [wait(ctx, t, timeout=300.0) for t in tickets]
        ctx.rb_serve_stop(True)
    U = np.stack([r[0] for r in res])
    assert np.all(info_b["status"] == 0)
    assert all(r[2]["status"] == 0 for r in res)
    for got in (u_b, U):
        for b, s in enumerate(sizes):
            assert rel(got[b, :s], u_or[b, :s]) <= TOL_MIXED, (b, s)
            assert np.all(got[b, s:] == 0.0)
