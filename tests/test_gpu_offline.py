"""The offline stage on the GPU (rb_offline_*: POD by the method of snapshots, Galerkin
projection, the trilinear tensor) against the oracle (oracle/offline.py) on the synthetic
high-fidelity model, and the reduced operators it makes solved online against the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import offline
from synth import hf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def signs(V, Vr, Z):
    """Signs s_j with s_j psi_j closest to the reference mode (modes are defined up to sign)."""
    return np.sign(np.einsum("jn,jn->j", V, (Z @ Vr.T).T))


@pytest.fixture(scope="module")
def case(rb):
    m = hf.make_hf_model(G=32, K=64, R=30, decay=0.85, q_c=2)
    n = 20
    lam_o, V_o = offline.pod(m.S, m.Z, n)
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        lam, V = ctx.rb_offline_pod(m.S, m.Z, n)
        A = [ctx.rb_offline_project(V, M) for M in m.A]
        f = np.stack([ctx.rb_offline_project_vector(V, fq) for fq in m.f])
        C = np.stack([ctx.rb_offline_tensor(V, t) for t in m.terms])
    return m, n, lam_o, V_o, lam, V, A, f, C


def test_pod_matches_oracle(rb, case):
    m, n, lam_o, V_o, lam, V, *_ = case
    # eigenvalues in decreasing order, to rounding of the largest
    assert np.all(np.diff(lam[:30]) <= 0)
    assert np.abs(lam[:n] - lam_o[:n]).max() <= 1e-12 * lam_o[0]
    np.testing.assert_allclose(V @ (m.Z @ V.T), np.eye(n), atol=1e-11)
    s = signs(V, V_o, m.Z)
    assert np.all(np.abs(s) == 1)
    d = V - s[:, None] * V_o
    err = np.sqrt(np.einsum("jn,jn->j", d, (m.Z @ d.T).T))
    # eigenvector accuracy of either side: eps lambda_max / gap
    lo = lam_o[: n + 1]
    below = lo[:n] - lo[1:]
    above = np.concatenate([[np.inf], lo[: n - 1] - lo[1:n]])
    gap = np.minimum(above, below)
    assert np.all(err <= 1e-12 * lam_o[0] / gap + 1e-12), (err, gap)


def test_projection_and_tensor_match_oracle(rb, case):
    m, n, lam_o, V_o, lam, V, A, f, C = case
    s = signs(V, V_o, m.Z)
    np.testing.assert_allclose(A[0], np.eye(n), atol=1e-11)   # the covariance matrix itself
    for M, Ag in zip(m.A, A):
        Ao = offline.project(V_o, M) * np.outer(s, s)
        np.testing.assert_allclose(Ag, Ao, atol=1e-9 * np.abs(Ao).max())
    for q in range(len(m.f)):
        fo = offline.project_vector(V_o, m.f[q]) * s
        np.testing.assert_allclose(f[q], fo, atol=1e-9 * np.abs(fo).max())
    for q in range(len(m.terms)):
        Co = offline.tensor(V_o, m.terms[q]) * np.einsum("j,l,k->jlk", s, s, s)
        scale = np.abs(Co).max()
        np.testing.assert_allclose(C[q], Co, atol=1e-9 * scale)
        np.testing.assert_allclose(C[q], -C[q].transpose(0, 2, 1), atol=1e-12 * scale)


def test_reduced_operators_solve_like_the_oracles(rb, case):
    """The reduced operators the GPU made, loaded into the online stage, give the oracle's
    solution on the oracle's reduced operators (signs of the modes aligned)."""
    m, n, lam_o, V_o, lam, V, A, f, C = case
    s = signs(V, V_o, m.Z)
    A = np.stack(A)
    # forcing scaled into the small-data regime of the reduced problem (input conditioning):
    # ||f|| <= lambda_min(A(mu))^2 / (4 sum_q ||C_q||_F) with lambda_min >= 1 / (2 Re_max)
    gamma = sum(np.linalg.norm(Cq) for Cq in C)
    lam_lo = 1.0 / (2 * 1000.0)
    factor = 0.25 * lam_lo ** 2 / (4 * gamma) / np.abs(f).sum(axis=1).max()
    fs = f * factor
    Ao = np.stack([offline.project(V_o, M) for M in m.A])
    Co = np.stack([offline.tensor(V_o, t) for t in m.terms])
    fo = np.stack([offline.project_vector(V_o, fq) for fq in m.f]) * factor
    g = np.random.default_rng(11)
    mu = np.stack([g.uniform(0, 35, 40), 10 ** g.uniform(2, 3, 40)], 1)
    o = oracle.Oracle(Ao, Co, fo)
    u_ref, _, inf_ref = o.solve(mu, threads=8)
    assert np.all(inf_ref["status"] == 0)
    for prec, tol in ((rb.RB_PREC_FP64, 1e-10), (rb.RB_PREC_MIXED, 1e-8)):
        with rb.Context(prec) as ctx:
            ctx.rb_load_operators(A, C, fs)
            u, _, info = ctx.rb_solve(mu)
        assert np.all(info["status"] == 0)
        err = np.linalg.norm(u * s[None, :] - u_ref, axis=1) / np.linalg.norm(u_ref, axis=1)
        assert err.max() <= tol, (prec, err.max())


def test_offline_argument_errors(rb):
    import scipy.sparse as sp
    with rb.Context() as ctx:
        Z = sp.identity(10, format="csr")
        with pytest.raises(rb.RbError):
            ctx.rb_offline_pod(np.ones((3, 10)), Z, 4)            # n > K
        with pytest.raises(rb.RbError):
            ctx.rb_offline_pod(np.ones((3, 10)), Z, 2)            # rank 1: lambda_2 = 0
        with pytest.raises(rb.RbError):
            ctx.rb_offline_pod(np.ones((rb.RB_POD_K_MAX + 1, 10)), Z, 2)
        bad = sp.csr_matrix((np.ones(1), (np.zeros(1), np.zeros(1))), shape=(10, 10))
        bad.indices[0] = 12                                        # column out of range
        with pytest.raises(rb.RbError):
            ctx.rb_offline_project(np.ones((2, 10)), bad)
