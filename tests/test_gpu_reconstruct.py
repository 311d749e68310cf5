"""GPU parity of pressure reconstruction with a combined basis (Sec. 4.2): p = sum_j u_j p^_j,
one batched product per query, against the oracle's plain loop; inside rb_solve (both
precisions) it replaces the recovery of Eq. sup-vvar."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def bound(P, u, n):
    """FP64 rounding bound of one sum of n products: n eps sum_j |P_kj u_j| (plus slack)."""
    out = np.empty((u.shape[0], P.shape[0]))
    for b in range(u.shape[0]):
        k = max(int(n[b]), 0)
        out[b] = 4 * max(k, 1) * 2.0 ** -52 * (np.abs(P[:, :k]) @ np.abs(u[b, :k]))
    return out


@pytest.mark.parametrize("n_max,m_r,nq", [(8, 30, 37), (50, 30, 4096), (120, 1000, 301),
                                          (300, 70001, 19)])
def test_reconstruct_parity(rb, n_max, m_r, nq):
    """Ragged query tiles (nq not a multiple of 8), coefficient tiles (m_r not a multiple of
    256), nested sizes, and rejected sizes (NaN rows)."""
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n_max, q_a=2, q_c=2, q_f=1)
    g = np.random.default_rng(n_max + m_r)
    P = g.standard_normal((m_r, n_max))
    u = g.standard_normal((nq, n_max))
    n = g.integers(1, n_max + 1, nq).astype(np.int32)
    n[:3] = [n_max, 0, n_max + 1]
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        ctx.rb_load_pressure_modes(P)
        p = ctx.rb_reconstruct_pressure(u, n)
        p_all = ctx.rb_reconstruct_pressure(u[:5])
    assert np.all(np.isnan(p[1])) and np.all(np.isnan(p[2]))
    ok = np.ones(nq, bool)
    ok[1:3] = False
    ref = oracle.reconstruct(P, u[ok], n[ok])
    assert np.all(np.abs(p[ok] - ref) <= bound(P, u[ok], n[ok]))
    ref5 = oracle.reconstruct(P, u[:5])
    assert np.all(np.abs(p_all - ref5) <= bound(P, u[:5], np.full(5, n_max)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_with_reconstruction(rb, prec):
    """rb_solve in reconstruction mode: the velocity as with recovery, p = P_hat u of it."""
    wl = synth.WORKLOADS["sweep_n50"]
    n_max = 40
    ops = synth.make_operators(wl, n_max=n_max)
    q = synth.make_queries(wl, batch=300, n_max=n_max)
    n = q.n.copy()
    n[::3] = 17  # nested truncations
    P = np.random.default_rng(3).standard_normal((25, n_max))
    P_ = rb.RB_PREC_FP64 if prec == "fp64" else rb.RB_PREC_MIXED
    with rb.Context(P_) as ctx:
        ctx.load_set(ops)
        u_rec, p_rec, _ = ctx.rb_solve(q.mu, n)
    with rb.Context(P_, pressure_method=rb.RB_PRESSURE_RECONSTRUCT) as ctx:
        ctx.load_set(ops)
        with pytest.raises(rb.RbError):
            ctx.rb_solve(q.mu, n)  # no modes loaded
        ctx.rb_load_pressure_modes(P)
        u, p, info = ctx.rb_solve(q.mu, n)
        p2 = ctx.rb_reconstruct_pressure(u, n)
        with pytest.raises(rb.RbError):
            ctx.rb_serve_start()  # the server only recovers
    assert np.all(info["status"] == 0)
    assert p.shape == (300, 25)
    np.testing.assert_allclose(u, u_rec, rtol=0, atol=1e-12 * np.abs(u_rec).max())
    np.testing.assert_array_equal(p, p2)
    ref = oracle.reconstruct(P, u, n)
    assert np.all(np.abs(p - ref) <= bound(P, u, n))
