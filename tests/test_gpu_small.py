"""The single-launch small-system solve of the mixed path (n_max <= 32, k_newton_small: one CTA
per query runs every Newton iteration) against the oracle, against the tensor-core pipeline, and
on the edge cases of the method (n = 1, nested sizes, caller-given theta, singular Jacobians,
the iteration cap, rejected sizes)."""
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


@pytest.mark.parametrize("n,nq", [(1, 5), (2, 40), (7, 33), (20, 300), (32, 150)])
def test_small_path_matches_oracle(rb, n, nq, monkeypatch):
    monkeypatch.setenv("RB_SMALL", "1")
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n)
    q = synth.make_queries(wl, batch=nq, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, inf_ref = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        ctx.rb_profile(True)
        u, p, info = ctx.rb_solve(mu)
        prof = ctx.rb_profile_read()
    assert prof["k_newton_small"][1] == 1  # one launch for the whole velocity solve
    assert prof.get("k_tc_gemm<sliced>", (0, 0))[1] == 0
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL_MIXED
    assert rel(p, p_ref).max() <= 10 * TOL_MIXED
    # quadratic convergence with an FP32 Jacobian: no more iterations than the exact Newton + 1
    assert np.all(info["iters"] <= inf_ref["iters"] + 1)


def test_small_path_equals_tensor_path(rb, monkeypatch):
    """The same batch through the tensor-core pipeline (RB_SMALL=0) and the single launch: both
    within the mixed tolerance of each other, sizes nested (1..24 of one n_max = 24 set)."""
    wl = synth.WORKLOADS["uneven_n120"]
    ops = synth.make_operators(wl, n_max=24, q_a=4, q_c=4)
    q = synth.make_queries(wl, batch=96, n_max=24)
    sizes = np.array([24, 1, 13, 20, 7, 24] * 16, dtype=np.int32)
    o = oracle.Oracle.from_set(ops)
    u_ref, _, _ = o.solve(q.mu, n=sizes, threads=8)
    res = {}
    for small in ("0", "1"):
        monkeypatch.setenv("RB_SMALL", small)
        with rb.Context(rb.RB_PREC_MIXED) as ctx:
            ctx.load_set(ops)
            res[small] = ctx.rb_solve(q.mu, n=sizes)
    for u, _, info in res.values():
        assert np.all(info["status"] == 0)
        assert rel(u, u_ref).max() <= TOL_MIXED
        for b, s in enumerate(sizes):
            assert np.all(u[b, s:] == 0.0)
    assert rel(res["0"][0], res["1"][0]).max() <= 2 * TOL_MIXED


def test_small_path_theta_and_statuses(rb, monkeypatch):
    monkeypatch.setenv("RB_SMALL", "1")
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=12)
    o = oracle.Oracle.from_set(ops)
    mu = np.array([[10.0, 200.0], [20.0, 300.0], [1.0, 900.0]])
    theta = np.stack([o.theta(*m) for m in mu])
    u_ref, _, _ = o.solve(mu, threads=4)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve_theta(theta)
    assert np.all(info["status"] == 0) and rel(u, u_ref).max() <= TOL_MIXED
    with rb.Context(rb.RB_PREC_MIXED, max_iter=1) as ctx:
        ctx.load_set(ops)
        _, _, info = ctx.rb_solve(mu, n=np.array([12, 0, 13], dtype=np.int32))
    assert info["status"][0] == rb.RB_Q_NOT_CONVERGED and info["iters"][0] == 1
    assert info["status"][1] == rb.RB_Q_REJECTED and info["status"][2] == rb.RB_Q_REJECTED
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.rb_load_operators(np.zeros_like(ops.A), np.zeros_like(ops.C), ops.f)
        _, _, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == rb.RB_Q_SINGULAR)


def test_single_query_manufactured_latency_path(rb):
    """The plain single query (n = 20, Q = 4, manufactured u* at mu0) takes the single launch by
    default and returns u* within the residual tolerance 1e-12 it is solved to."""
    ops = synth.make_operators(synth.WORKLOADS["single_n20"])
    oracle.manufacture(ops, (10.0, 200.0))
    with rb.Context(rb.RB_PREC_MIXED, tol_res=1e-12) as ctx:
        ctx.load_set(ops)
        ctx.rb_profile(True)
        u, _, info = ctx.rb_solve(np.array([[10.0, 200.0]]))
        prof = ctx.rb_profile_read()
    assert prof["k_newton_small"][1] == 1
    assert info["status"][0] == 0
    assert rel(u[0], ops.u_star) <= 1e-11
