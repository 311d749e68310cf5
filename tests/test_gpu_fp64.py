"""GPU parity of the FP64 path against the FP64 CPU oracle, through the C ABI.

Tolerance: relative L2 error <= 1e-10 per query on the velocity (and 1e-9 on the pressure,
whose recovery amplifies the velocity error by ||B^-1|| ||As||), the bound stated for FP64 paths.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


def small_set(n, q_a=3, q_c=3, q_f=2, q_b=0, m=0, c_dtype="f64", wid=80, manufactured=False):
    wl = synth.Workload("t", wid, n_max=n, q_a=q_a, q_c=q_c, q_f=q_f, q_b=q_b, m=m,
                        c_dtype=c_dtype, manufactured=manufactured,
                        mu0=(10.0, 200.0) if manufactured else None,
                        re_range=(200.0, 200.0) if manufactured else (100.0, 1000.0))
    return synth.make_operators(wl)


def test_manufactured_single_n20(rb):
    ops = synth.make_operators(synth.WORKLOADS["single_n20"])
    oracle.manufacture(ops, (10.0, 200.0))
    with rb.Context(rb.RB_PREC_FP64, tol_res=1e-12) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(np.array([[10.0, 200.0]]))
    assert info["status"][0] == rb.RB_Q_OK
    assert rel(u[0], ops.u_star) <= 1e-12
    o = oracle.Oracle.from_set(ops)
    u_ref, _, info_ref = o.solve(np.array([[10.0, 200.0]]), tol_res=1e-12)
    assert rel(u[0], u_ref[0]) <= TOL64
    assert info["iters"][0] == info_ref["iters"][0]


def test_manufactured_pressure(rb):
    ops = small_set(14, q_a=4, q_c=4, q_f=2, q_b=3, m=9, wid=81, manufactured=True)
    oracle.manufacture(ops, (10.0, 200.0))
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(np.array([[10.0, 200.0]]))
    assert info["status"][0] == 0
    assert rel(u[0], ops.u_star) <= 1e-12
    assert rel(p[0], ops.p_star) <= 1e-10


@pytest.mark.parametrize("n", [1, 2, 7, 33, 50])
def test_sweep_parity(rb, n):
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n)
    q = synth.make_queries(wl, batch=61, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, inf_ref = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0) and np.all(inf_ref["status"] == 0)
    assert rel(u, u_ref).max() <= TOL64
    assert rel(p, p_ref).max() <= 10 * TOL64
    assert np.all(np.abs(info["iters"] - inf_ref["iters"]) <= 1)


def test_nested_truncation_mixed_sizes(rb):
    """Queries of several sizes in one call; each equals the oracle on its leading blocks."""
    wl = synth.WORKLOADS["uneven_n120"]
    ops = synth.make_operators(wl, n_max=40, q_a=4, q_c=4)
    mu = synth.make_queries(wl, batch=40).mu
    sizes = np.array([1, 5, 17, 20, 39, 40] * 7)[:40].astype(np.int32)
    o = oracle.Oracle.from_set(ops)
    u_ref, _, inf_ref = o.solve(mu, n=sizes, threads=8)
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(mu, n=sizes)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL64
    for b, n in enumerate(sizes):
        assert np.all(u[b, n:] == 0.0)


def test_fp32_storage_and_theta_user(rb):
    ops = small_set(24, q_a=4, q_c=5, q_f=3, c_dtype="f32", wid=82)
    o = oracle.Oracle.from_set(ops)
    g = np.random.default_rng(0)
    mu = np.stack([g.uniform(0, 35, 16), 10 ** g.uniform(2, 3, 16)], 1)
    theta = np.stack([o.theta(*m) for m in mu])
    u_ref, _, _ = o.solve_theta(theta)
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve_theta(theta)
        u2, _, _ = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL64
    assert rel(u2, u_ref).max() <= TOL64


def test_eval_residual_and_jacobian(rb):
    n = 37
    ops = small_set(n, q_a=3, q_c=4, wid=83)
    o = oracle.Oracle.from_set(ops)
    g = np.random.default_rng(1)
    mu = np.stack([g.uniform(0, 35, 9), 10 ** g.uniform(2, 3, 9)], 1)
    u = g.standard_normal((9, n)) * 0.05
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        R, J = ctx.rb_eval(mu, n, u, rb.RB_PREC_FP64)
    for b in range(9):
        th = o.theta(*mu[b])
        Rr = o.residual(n, th, u[b])
        Jr = o.jacobian(n, th, u[b])
        A, f = o.assemble(n, th)
        scale = np.abs(A).sum(1) @ np.abs(u[b]) + np.linalg.norm(f)
        assert np.linalg.norm(R[b] - Rr) <= 1e-13 * scale
        assert np.abs(J[b] - Jr).max() <= 1e-13 * np.abs(Jr).max()


@pytest.mark.parametrize("n", [1, 3, 64, 130])
def test_gepp(rb, n):
    g = np.random.default_rng(n)
    M = g.standard_normal((5, n, n))
    M[1, 0, :] = 0.0
    M[1, :, 0] = 0.0  # singular
    rhs = g.standard_normal((5, n))
    with rb.Context() as ctx:
        x, st = ctx.rb_gepp_solve(M, rhs)
    for b in range(5):
        Mb, xb = M[b].copy(), rhs[b].copy()
        sing = oracle.lib().oracle_gepp_solve(n, Mb.ctypes.data, xb.ctypes.data)
        assert (st[b] != 0) == (sing != 0)
        if not sing:
            np.testing.assert_allclose(x[b], xb, rtol=1e-9, atol=1e-12)


def test_status_codes(rb):
    ops = small_set(6, wid=84)
    mu = np.array([[10.0, 200.0], [20.0, 300.0]])
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.rb_load_operators(np.zeros_like(ops.A), np.zeros_like(ops.C), ops.f)
        _, _, info = ctx.rb_solve(mu)
        assert np.all(info["status"] == rb.RB_Q_SINGULAR)
        A = ops.A.copy()
        A[0, 0, 0] = np.nan
        ctx.rb_load_operators(A, ops.C, ops.f)
        _, _, info = ctx.rb_solve(mu)
        assert np.all(info["status"] == rb.RB_Q_NONFINITE)
    with rb.Context(rb.RB_PREC_FP64, max_iter=1) as ctx:
        ctx.load_set(ops)
        _, _, info = ctx.rb_solve(mu)
        assert np.all(info["status"] == rb.RB_Q_NOT_CONVERGED) and np.all(info["iters"] == 1)
        u, _, info = ctx.rb_solve(mu, n=np.array([0, 7], dtype=np.int32))
        assert np.all(info["status"] == rb.RB_Q_REJECTED) and np.all(u == 0)


def test_empty_and_argument_errors(rb):
    ops = small_set(5, wid=85)
    with rb.Context() as ctx:
        with pytest.raises(rb.RbError):
            ctx.rb_solve(np.zeros((1, 2)))           # no operators yet
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(np.zeros((0, 2)))
        assert u.shape == (0, 5)
        with pytest.raises(rb.RbError):
            ctx.rb_load_operators(np.zeros((1, 400, 400)), np.zeros((1, 1, 1, 1)), np.zeros((1, 400)))


@pytest.mark.parametrize("n,q", [(160, 2), (300, 2)])
def test_large_n_sampled(rb, n, q):
    """Jacobian in shared memory up to the limit, in global scratch beyond it."""
    wl = synth.WORKLOADS["dense_n300"]
    ops = synth.make_operators(wl, n_max=n, q_a=q, q_c=q, q_f=2)
    mu = synth.corner_queries(wl)[:2]
    o = oracle.Oracle.from_set(ops)
    u_ref, _, inf_ref = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL64


def test_full_sweep_batch_sampled(rb):
    """The n = 50 sweep at its full batch (4096 queries, one launch), checked on a stratified
    sample of 64 queries plus the corners of the parameter box."""
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0)
    idx = np.concatenate([np.argsort(mu[:-4, 1])[:: len(mu) // 60][:60], np.arange(len(mu) - 4, len(mu))])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(mu[idx], threads=16)
    assert rel(u[idx], u_ref).max() <= TOL64
    assert rel(p[idx], p_ref).max() <= 10 * TOL64
