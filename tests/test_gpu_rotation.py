"""GPU parity for the polynomial parameter family: the monomials phi^q of the rotation angle
that the truncated rotation series of Sec. 5 (Eq. rotsum) makes the affine coefficients of
every pulled-back form. Q_a = 50, Q_c = 49, Q_f = 50, Q_b = 48 (12 series terms); the FP64 and
mixed paths, rb_solve against rb_solve_theta, and the server, all against the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-8


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


@pytest.fixture(scope="module", params=[20, 50])
def rotation(request):
    n = request.param
    wl = synth.WORKLOADS["rotation_n50"]
    ops = synth.make_operators(wl, n_max=n)
    q = synth.make_queries(wl, batch=260, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl), [[-30.0, 150.0], [0.0, 500.0]]])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, info_ref = o.solve(mu, threads=8)
    assert np.all(info_ref["status"] == 0)
    return wl, ops, mu, o, u_ref, p_ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rotation_parity(rb, rotation, prec):
    wl, ops, mu, o, u_ref, p_ref = rotation
    P = rb.RB_PREC_FP64 if prec == "fp64" else rb.RB_PREC_MIXED
    tol = TOL_FP64 if prec == "fp64" else TOL_MIXED
    with rb.Context(P, theta_family=rb.RB_THETA_POLY) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0), np.unique(info["status"], return_counts=True)
    assert rel(u, u_ref).max() <= tol
    assert rel(p, p_ref).max() <= 10 * tol


def test_rotation_theta_rows_match(rb, rotation):
    """theta evaluated on the device equals the oracle's rows passed in by the caller."""
    wl, ops, mu, o, u_ref, p_ref = rotation
    th = np.stack([o.theta(*m) for m in mu])
    with rb.Context(rb.RB_PREC_FP64, theta_family=rb.RB_THETA_POLY) as ctx:
        ctx.load_set(ops)
        u1, p1, _ = ctx.rb_solve(mu)
        u2, p2, i2 = ctx.rb_solve_theta(th)
    assert np.all(i2["status"] == 0)
    assert rel(u1, u2).max() <= 1e-12 and rel(p1, p2).max() <= 1e-11


def test_family_mismatch_is_refused(rb, rotation):
    wl, ops, *_ = rotation
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        with pytest.raises(ValueError):
            ctx.load_set(ops)


def test_rotation_server(rb, rotation):
    wl, ops, mu, o, u_ref, p_ref = rotation
    with rb.Context(rb.RB_PREC_MIXED, theta_family=rb.RB_THETA_POLY) as ctx:
        ctx.load_set(ops)
        ctx.rb_serve_start()
        tickets = [ctx.rb_serve_submit(m) for m in mu[:64]]
        res = []
        for t in tickets:
            t0 = time.time()
            while True:
                r = ctx.rb_serve_poll(t)
                if r is not None:
                    res.append(r)
                    break
                assert time.time() - t0 < 60.0
                time.sleep(1e-4)
        ctx.rb_serve_stop(True)
    U = np.stack([r[0] for r in res])
    P = np.stack([r[1] for r in res])
    assert all(r[2]["status"] == 0 for r in res)
    assert rel(U, u_ref[:64]).max() <= TOL_MIXED
    assert rel(P, p_ref[:64]).max() <= 10 * TOL_MIXED
