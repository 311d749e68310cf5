"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the mathematics.

Each test ties one piece of the oracle to something other than its own code: a hand-derived
closed-form case, the manufactured solution, the skew identity of the solenoidal convection
form, the Euler identity of the quadratic term, a finite-difference Jacobian (exact for a
quadratic residual), the C = 0 reduction to one linear solve, quadratic Newton convergence,
nested truncation, the n = 1 closed form, and elimination against LAPACK.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_set(n=8, q_a=3, q_c=3, q_f=2, q_b=0, m=0, c_dtype="f64", manufactured=False,
              wid=90, re_range=(100.0, 1000.0)):
    wl = synth.Workload("test", wid, n_max=n, q_a=q_a, q_c=q_c, q_f=q_f, q_b=q_b, m=m,
                        c_dtype=c_dtype, manufactured=manufactured, re_range=re_range,
                        mu0=(10.0, 200.0) if manufactured else None)
    return synth.make_operators(wl)


def test_theta_closed_forms(oracle_lib):
    ops = small_set(n=3, q_a=4, q_c=4, q_f=4)
    o = oracle_lib.Oracle.from_set(ops)
    # alpha = 0: sin terms vanish, cos terms are 1; theta^a carries 1/Re (Sec. 2.4 split)
    t = o.theta(0.0, 250.0)
    np.testing.assert_allclose(t[:4], [1 / 250.0, 0.0, 1 / 250.0, 0.0], atol=1e-18)
    np.testing.assert_allclose(t[4:8], [1.0, 0.0, 1.0, 0.0], atol=1e-15)
    # alpha = 90 deg: trig = (1, sin 90, cos 180, sin 270) = (1, 1, -1, -1)
    t = o.theta(90.0, 1.0)
    np.testing.assert_allclose(t[4:8], [1.0, 1.0, -1.0, -1.0], atol=1e-15)
    np.testing.assert_allclose(t[8:12], [1.0, 1.0, -1.0, -1.0], atol=1e-15)


def _rotation_series_set(q, m=2):
    """Operators whose q-th terms are J^q / q! with J the 2 x 2 rotation generator, so that
    sum_q phi^q J^q / q! is the rotation matrix R(phi) (Sec. 5, Eq. rotsum)."""
    J = np.array([[0.0, -1.0], [1.0, 0.0]])
    P = [np.linalg.matrix_power(J, k) / math.factorial(k) for k in range(q)]
    A = np.stack(P)
    f = np.stack([Pk @ np.array([1.0, 0.0]) for Pk in P])
    C = np.zeros((1, 2, 2, 2))
    B = np.stack(P)
    As = np.zeros((q, m, 2))
    Cs = np.zeros((1, 2, 2, m))
    return A, C, f, B, As, Cs, f.copy()


@pytest.mark.parametrize("alpha", [0.0, 7.5, 35.0, -20.0])
def test_poly_theta_is_rotation_series(oracle_lib, alpha):
    # Polynomial family: theta_q = phi^q (theta^a_q = phi^q / Re). With operators J^q / q! the
    # assembled A(mu) and f(mu) are the rotation R(phi) / Re and R(phi) e_0, the closed form of
    # the exponential series; 30 terms leave a truncation error below 1e-30.
    A, C, f, B, As, Cs, fs = _rotation_series_set(30)
    o = oracle_lib.Oracle(A, C, f, B, As, Cs, fs, theta_family=2)
    re = 300.0
    phi = math.radians(alpha)
    t = o.theta(alpha, re)
    Am, fm = o.assemble(2, t)
    R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    np.testing.assert_allclose(Am, R / re, rtol=0, atol=1e-17)
    np.testing.assert_allclose(fm, R[:, 0], rtol=0, atol=1e-15)
    # pressure with u = 0: B(mu) p = fs(mu) is R(phi) p = R(phi) e_0, so p = e_0
    p, rc = o.pressure(2, t, np.zeros(2))
    assert rc == 0
    np.testing.assert_allclose(p, [1.0, 0.0], rtol=0, atol=1e-14)


def test_rotation_pin_detects_shifted_powers(oracle_lib):
    """The rotation pin is sensitive: a θ row with every power shifted by one (φ^(q+1)) or with
    1/Re left off θᵃ assembles something other than R(φ)/Re."""
    A, C, f, B, As, Cs, fs = _rotation_series_set(30)
    o = oracle_lib.Oracle(A, C, f, B, As, Cs, fs, theta_family=2)
    phi, re = math.radians(20.0), 300.0
    R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    good = o.theta(20.0, re)
    shifted = good.copy()
    shifted[:30] = [phi ** (q + 1) / re for q in range(30)]
    no_re = good.copy()
    no_re[:30] *= re
    for t in (shifted, no_re):
        Am, _ = o.assemble(2, t)
        assert np.abs(Am - R / re).max() > 1e-4


def test_poly_theta_monomials(oracle_lib):
    ops = small_set(n=3, q_a=4, q_c=4, q_f=4)
    o = oracle_lib.Oracle(ops.A, ops.C, ops.f, theta_family=2)
    # alpha = 0: only the constant monomial survives
    t = o.theta(0.0, 250.0)
    np.testing.assert_array_equal(t[:4], [1 / 250.0, 0.0, 0.0, 0.0])
    np.testing.assert_array_equal(t[4:12], [1.0, 0.0, 0.0, 0.0] * 2)
    # alpha = 180 / pi degrees: phi = 1, every monomial is 1
    t = o.theta(180.0 / math.pi, 1.0)
    np.testing.assert_allclose(t, np.ones(12), rtol=1e-15)
    # alpha = -90 deg: phi = -pi/2, signs alternate
    t = o.theta(-90.0, 1.0)
    np.testing.assert_allclose(t[4:8], [(-math.pi / 2) ** k for k in range(4)], rtol=1e-15)


def _golden_set():
    with open(os.path.join(GOLDEN, "n2_closed_form.json")) as fh:
        g = json.load(fh)
    n, m = g["n"], g["m"]
    C = np.zeros((1, n, n, n))
    for q, j, l, k, v in g["C_nonzero"]:
        C[q, j, l, k] = v
    Cs = np.zeros((1, n, n, m))
    for q, j, l, k, v in g["Cs_nonzero"]:
        Cs[q, j, l, k] = v
    return g, C, Cs


def test_golden_n2_closed_form(oracle_lib):
    g, C, Cs = _golden_set()
    o = oracle_lib.Oracle(np.array(g["A"]), C, np.array(g["f"]), np.array(g["B"]),
                          np.array(g["As"]), Cs, np.array(g["fs"]))
    u, p, info = o.solve(np.array([g["mu"]]), tol_upd=1e-14, tol_res=1e-14)
    assert info["status"][0] == oracle_lib.Q_OK
    np.testing.assert_allclose(u[0], g["u"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(p[0], g["p"], rtol=0, atol=1e-13)


def test_manufactured_solution(oracle_lib):
    """P1: with f_0 built from u* at mu0, Newton from u = 0 returns u* (and p*)."""
    ops = small_set(n=12, q_a=4, q_c=4, q_f=2, q_b=3, m=7, manufactured=True, wid=91,
                    re_range=(200.0, 200.0))
    oracle_lib.manufacture(ops, (10.0, 200.0))
    # the manufactured forcing is also checked by an independent restatement here
    o = oracle_lib.Oracle.from_set(ops)
    th = o.theta(10.0, 200.0)
    ta, tc, tf = th[:4], th[4:8], th[8:10]
    us = ops.u_star
    r = (np.einsum("q,qkj,j->k", ta, ops.A, us)
         + np.einsum("q,qjlk,j,l->k", tc, ops.C, us, us)
         - np.einsum("q,qk->k", tf, ops.f))
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(ops.f[0])
    u, p, info = o.solve(np.array([[10.0, 200.0]]), tol_upd=1e-10, tol_res=1e-12)
    assert info["status"][0] == oracle_lib.Q_OK
    assert np.linalg.norm(u[0] - us) <= 1e-12 * np.linalg.norm(us)
    assert np.linalg.norm(p[0] - ops.p_star) <= 1e-11 * np.linalg.norm(ops.p_star)


def test_manufactured_single_n20(oracle_lib):
    """P1 on the plain single-query workload (n = 20, Q = 4, mu0 = (10 deg, Re 200))."""
    ops = synth.make_operators(synth.WORKLOADS["single_n20"])
    oracle_lib.manufacture(ops, (10.0, 200.0))
    o = oracle_lib.Oracle.from_set(ops)
    u, _, info = o.solve(np.array([[10.0, 200.0]]), tol_upd=1e-10, tol_res=1e-12)
    assert info["status"][0] == oracle_lib.Q_OK
    assert np.linalg.norm(u[0] - ops.u_star) <= 1e-12 * np.linalg.norm(ops.u_star)
    assert info["iters"][0] >= 3


@pytest.mark.parametrize("c_dtype", ["f64", "f32"])
def test_skew_and_energy_identity(oracle_lib, c_dtype):
    """P2: u^T Cmu(u, u) = 0 for C skew in its last two indices; so u^T R = u^T A u - u^T f."""
    ops = small_set(n=10, c_dtype=c_dtype)
    o = oracle_lib.Oracle.from_set(ops)
    g = np.random.default_rng(5)
    for _ in range(5):
        th = o.theta(g.uniform(0, 35), 10 ** g.uniform(2, 3))
        u = g.standard_normal(10)
        cv = o.convection(10, th, u)
        scale = np.sum(np.abs(ops.C)) * np.max(np.abs(u)) ** 3
        assert abs(u @ cv) <= 1e-14 * scale
        A, f = o.assemble(10, th)
        R = o.residual(10, th, u)
        assert abs(u @ R - (u @ A @ u - u @ f)) <= 1e-13 * (abs(u @ A @ u) + abs(u @ f) + scale)


def test_skew_identity_detects_wrong_pair(oracle_lib):
    """The skew identity fails when the tensor's test index is not the last one."""
    ops = small_set(n=10)
    C_wrong = np.ascontiguousarray(ops.C.transpose(0, 2, 3, 1))  # test index moved to front
    o = oracle_lib.Oracle(ops.A, C_wrong, ops.f)
    th = o.theta(20.0, 300.0)
    u = np.random.default_rng(3).standard_normal(10)
    cv = o.convection(10, th, u)
    assert abs(u @ cv) > 1e-6 * np.linalg.norm(cv) * np.linalg.norm(u)


@pytest.mark.parametrize("skew", [True, False])
def test_euler_identity(oracle_lib, skew):
    """P3: the convection Jacobian applied to u is twice the convection term (any C)."""
    n = 9
    ops = small_set(n=n)
    C = ops.C if skew else np.random.default_rng(11).standard_normal(ops.C.shape)
    o = oracle_lib.Oracle(ops.A, C, ops.f)
    th = o.theta(17.0, 420.0)
    u = np.random.default_rng(4).standard_normal(n)
    A, _ = o.assemble(n, th)
    Jc = o.jacobian(n, th, u) - A
    cv = o.convection(n, th, u)
    np.testing.assert_allclose(Jc @ u, 2 * cv, rtol=0, atol=1e-12 * np.abs(Jc).sum())


@pytest.mark.parametrize("n,skew", [(2, True), (3, False), (4, True), (6, False)])
def test_fd_jacobian_exact(oracle_lib, n, skew):
    """P5: R is quadratic in u, so the central difference equals the Jacobian column up to
    rounding, for every h."""
    ops = small_set(n=n, wid=92 + n)
    C = ops.C if skew else np.random.default_rng(n).standard_normal(ops.C.shape)
    o = oracle_lib.Oracle(ops.A, C, ops.f)
    th = o.theta(23.0, 150.0)
    u = np.random.default_rng(7).standard_normal(n)
    J = o.jacobian(n, th, u)
    h = 0.5
    Jfd = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        Jfd[:, j] = (o.residual(n, th, u + e) - o.residual(n, th, u - e)) / (2 * h)
    assert np.max(np.abs(J - Jfd)) <= 1e-12 * np.max(np.abs(J))


def test_c_zero_reduces_to_linear_solve(oracle_lib):
    """P4: with C = 0 one Newton step gives A(mu)^-1 f(mu); the next update is ~0."""
    ops = small_set(n=15)
    o = oracle_lib.Oracle(ops.A, np.zeros_like(ops.C), ops.f)
    mu = (12.0, 333.0)
    th = o.theta(*mu)
    A, f = o.assemble(15, th)
    u, info, tr, tu = o.newton(15, th, tol_upd=1e-10, tol_res=1e-10)
    x = np.linalg.solve(A, f)
    assert info.status == 0 and info.iters == 2
    assert np.linalg.norm(u - x) <= 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(tu[0] - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)


def test_quadratic_convergence(oracle_lib):
    """P6: ||delta_{k+1}|| <= K ||delta_k||^2 while above the rounding floor."""
    ops = synth.make_operators(synth.WORKLOADS["sweep_n50"], n_max=30)
    # viscous terms weakened 64x so that several iterations are in the quadratic phase
    o = oracle_lib.Oracle(ops.A / 64.0, ops.C, ops.f)
    th = o.theta(35.0, 1000.0)
    u, info, tr, tu = o.newton(30, th, tol_upd=1e-13, tol_res=1e-13)
    assert info.status == 0 and info.iters >= 5
    ks = [tu[k + 1] / tu[k] ** 2 for k in range(len(tu) - 1) if tu[k + 1] > 1e-12 * tu[0]]
    assert len(ks) >= 3, "no quadratic phase observed"
    assert max(ks) <= 4 * min(ks)
    # the ratio of successive updates falls (superlinear), unlike a linear rate
    rs = [tu[k + 1] / tu[k] for k in range(len(tu) - 1) if tu[k + 1] > 1e-12 * tu[0]]
    assert all(rs[i + 1] < rs[i] for i in range(len(rs) - 1))


def test_truncation_invariance(oracle_lib):
    """P7: a size-n query on the n_max set equals the oracle on the extracted leading blocks."""
    ops = small_set(n=14, q_b=2, m=5)
    o = oracle_lib.Oracle.from_set(ops)
    n = 9
    mu = np.array([[21.0, 640.0]])
    u, p, info = o.solve(mu, n=np.array([n]))
    o2 = oracle_lib.Oracle(ops.A[:, :n, :n], ops.C[:, :n, :n, :n], ops.f[:, :n], ops.B,
                           ops.As[:, :, :n], ops.Cs[:, :n, :n, :], ops.fs)
    u2, p2, info2 = o2.solve(mu)
    assert info["status"][0] == 0 and info2["status"][0] == 0
    np.testing.assert_array_equal(u[0, :n], u2[0])
    np.testing.assert_array_equal(u[0, n:], 0.0)
    np.testing.assert_array_equal(p[0], p2[0])


def test_n1_closed_form(oracle_lib):
    """P8: for n = 1 a skew C vanishes and u = f(mu) / a(mu)."""
    ops = small_set(n=1, q_a=2, q_c=2, q_f=2)
    assert np.all(ops.C == 0)
    o = oracle_lib.Oracle.from_set(ops)
    th = o.theta(30.0, 500.0)
    u, info, _, _ = o.newton(1, th)
    a = th[0] * ops.A[0, 0, 0] + th[1] * ops.A[1, 0, 0]
    f = th[4] * ops.f[0, 0] + th[5] * ops.f[1, 0]
    assert info.status == 0
    assert abs(u[0] - f / a) <= 1e-15 * abs(f / a)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40])
def test_gepp_matches_lapack(oracle_lib, n):
    g = np.random.default_rng(n)
    M = g.standard_normal((n, n))
    b = g.standard_normal(n)
    x = b.copy()
    Mc = M.copy()
    assert oracle_lib.lib().oracle_gepp_solve(n, Mc.ctypes.data, x.ctypes.data) == 0
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)


def test_gepp_needs_pivoting_and_detects_singular(oracle_lib):
    M = np.array([[0.0, 1.0], [1.0, 0.0]])
    x = np.array([2.0, 3.0])
    assert oracle_lib.lib().oracle_gepp_solve(2, M.ctypes.data, x.ctypes.data) == 0
    np.testing.assert_array_equal(x, [3.0, 2.0])
    S = np.array([[1.0, 2.0], [2.0, 4.0]])
    y = np.array([1.0, 1.0])
    assert oracle_lib.lib().oracle_gepp_solve(2, S.ctypes.data, y.ctypes.data) == 1


def test_pressure_linear_reduction(oracle_lib):
    """With As = 0 and Cs = 0 the recovery is B(mu)^-1 fs(mu) (LAPACK)."""
    ops = small_set(n=6, q_b=3, m=5)
    o = oracle_lib.Oracle(ops.A, ops.C, ops.f, ops.B, np.zeros_like(ops.As),
                          np.zeros_like(ops.Cs), ops.fs)
    th = o.theta(5.0, 120.0)
    u = np.random.default_rng(1).standard_normal(6)
    p, rc = o.pressure(6, th, u)
    tb, tf = th[3 + 3 + 2:], th[3 + 3:3 + 3 + 2]
    Bm = np.tensordot(tb, ops.B, axes=1)
    fs = np.tensordot(tf, ops.fs, axes=1)
    np.testing.assert_allclose(p, np.linalg.solve(Bm, fs), rtol=1e-12)


def test_status_singular_and_nonfinite(oracle_lib):
    ops = small_set(n=5)
    o = oracle_lib.Oracle(np.zeros_like(ops.A), np.zeros_like(ops.C), ops.f)
    u, _, info = o.solve(np.array([[10.0, 200.0]]))
    assert info["status"][0] == oracle_lib.Q_SINGULAR
    A = ops.A.copy()
    A[0, 0, 0] = np.nan
    o = oracle_lib.Oracle(A, ops.C, ops.f)
    u, _, info = o.solve(np.array([[10.0, 200.0]]))
    assert info["status"][0] in (oracle_lib.Q_NONFINITE, oracle_lib.Q_SINGULAR)
    o = oracle_lib.Oracle.from_set(ops)
    u, _, info = o.solve(np.array([[10.0, 200.0]]), max_iter=1)
    assert info["status"][0] == oracle_lib.Q_NOT_CONVERGED and info["iters"][0] == 1


def test_sweep_workload_converges(oracle_lib):
    """Every query of a sample of the n = 50 sweep converges from u = 0 (unique regime)."""
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl, batch=16)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle_lib.Oracle.from_set(ops)
    u, p, info = o.solve(mu, threads=4)
    assert np.all(info["status"] == 0), info
    assert np.all(info["iters"] <= 15)
    assert np.all(np.isfinite(p))


def test_rotation_workload_converges(oracle_lib):
    """The polynomial-family workload (Sec. 5 rotation series) converges from u = 0, and its
    theta row equals the one the trigonometric row of the same angle would give for phi = 0."""
    wl = synth.WORKLOADS["rotation_n50"]
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl, batch=12)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle_lib.Oracle.from_set(ops)
    u, p, info = o.solve(mu, threads=4)
    assert np.all(info["status"] == 0), info
    assert np.all(info["iters"] <= 15)
    assert np.all(np.isfinite(p))
    # at alpha = 0 both families reduce to (1/Re, 0, ..., | 1, 0, ... | ...)
    t_poly = o.theta(0.0, 500.0)
    t_trig = oracle_lib.Oracle(ops.A, ops.C, ops.f, ops.B, ops.As, ops.Cs, ops.fs).theta(0.0, 500.0)
    nz = np.nonzero(t_poly)[0]
    np.testing.assert_array_equal(nz, [0, wl.q_a, wl.q_a + wl.q_c, wl.q_a + wl.q_c + wl.q_f])
    np.testing.assert_array_equal(t_poly[nz], t_trig[nz])


def test_reconstruct_unit_vectors_and_truncation(oracle_lib):
    """Pressure reconstruction (Sec. 4.2): u = e_j gives column j of P_hat exactly (the pressure
    data of basis function j); columns from n on are never read (NaN there stays out)."""
    g = np.random.default_rng(5)
    P = g.standard_normal((7, 5))
    for j in range(5):
        e = np.zeros(5)
        e[j] = 1.0
        np.testing.assert_array_equal(oracle_lib.reconstruct(P, e)[0], P[:, j])
    Pn = P.copy()
    Pn[:, 3:] = np.nan
    u = g.standard_normal(5)
    p = oracle_lib.reconstruct(Pn, u, n=[3])[0]
    brute = [math.fsum(P[k, j] * u[j] for j in range(3)) for k in range(7)]
    np.testing.assert_allclose(p, brute, rtol=1e-15, atol=1e-15)


def test_combined_basis_reproduces_its_snapshots(oracle_lib):
    """Second construction of Sec. 4.2: POD of the velocity snapshots (method of snapshots,
    Sec. 3.2), the pressure functions combined with the same snapshot coefficients. With as many
    independent snapshots as modes, reconstructing a snapshot from its coefficients in the POD
    basis returns that snapshot's own pressure."""
    g = np.random.default_rng(11)
    K, n_h, m_h = 6, 9, 4                  # snapshots, velocity / pressure dofs
    U = g.standard_normal((K, n_h))        # velocity snapshots (rows)
    Pp = g.standard_normal((K, m_h))       # their pressures
    lam, W = np.linalg.eigh(U @ U.T)       # correlation matrix of the snapshots
    V = W / np.sqrt(lam)[None, :]          # coefficient vectors v^j (columns)
    Psi = U.T @ V                          # orthonormal velocity modes psi_j = sum_i v^j_i u_i
    np.testing.assert_allclose(Psi.T @ Psi, np.eye(K), atol=1e-12)
    P_hat = Pp.T @ V                       # p^_j = sum_i v^j_i p_i, column j
    for i in range(K):
        eta = Psi.T @ U[i]                 # velocity coefficients of snapshot i
        np.testing.assert_allclose(oracle_lib.reconstruct(P_hat, eta)[0], Pp[i], atol=1e-11)
