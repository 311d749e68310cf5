"""Pins of the offline-stage oracle (oracle/offline.py) to facts outside itself: the identities
of POD by the method of snapshots (Sec. 3.2), the Galerkin projection of the covariance's own
matrix (Sec. 3.5), and the tensor of Sec. 3.6 against the high-fidelity trilinear form evaluated
by its definition with explicit loops over the grid (no sparse matrices)."""
import numpy as np
import pytest

from oracle import offline
from synth import hf


@pytest.fixture(scope="module")
def model():
    return hf.make_hf_model(G=12, K=40, R=24, decay=0.8, q_c=2)


def test_modes_are_orthonormal_in_the_covariance(model):
    lam, V = offline.pod(model.S, model.Z, 16)
    assert np.all(np.diff(lam[:24]) <= 0)  # decreasing
    np.testing.assert_allclose(V @ (model.Z @ V.T), np.eye(16), atol=1e-11)


def test_pod_optimality_identities(model):
    """sum_i ||phi_i||_z^2 = sum_k lambda_k, and the projection error of the snapshots onto the
    first n modes is the sum of the remaining eigenvalues (Sec. 3.2, after Eq. spd)."""
    S, Z = model.S, model.Z
    lam, V = offline.pod(S, Z, 10)
    energy = np.einsum("kn,kn->", S, (Z @ S.T).T)
    assert abs(energy - lam.sum()) <= 1e-11 * energy
    coef = S @ (Z @ V.T)                 # z(phi_i, psi_j)
    err = S - coef @ V                   # phi_i - P_V phi_i
    e2 = np.einsum("kn,kn->", err, (Z @ err.T).T)
    assert abs(e2 - lam[10:].sum()) <= 1e-9 * energy


def test_planted_subspace_is_recovered(model):
    """The snapshots are combinations of R fields: with n = R modes every snapshot is reproduced
    and the eigenvalues past R vanish (to rounding)."""
    S, Z = model.S, model.Z
    R = 24
    lam, V = offline.pod(S, Z, R)
    assert lam[R:].max() <= 1e-12 * lam[0]
    coef = S @ (Z @ V.T)
    np.testing.assert_allclose(coef @ V, S, atol=1e-10 * np.abs(S).max())


def test_projection_of_the_covariance_matrix_is_the_identity(model):
    """A_0 is the H1 stiffness, the covariance matrix itself: its Galerkin projection onto
    z-orthonormal modes is the identity (Eq. redorth-final)."""
    _, V = offline.pod(model.S, model.Z, 12)
    np.testing.assert_allclose(offline.project(V, model.A[0]), np.eye(12), atol=1e-11)
    # the mass matrix projects to a symmetric positive definite matrix
    M = offline.project(V, model.A[1])
    np.testing.assert_allclose(M, M.T, atol=1e-16)
    assert np.linalg.eigvalsh(M).min() > 0


def brute_form(G, omega, a, v, w):
    """c(a, v, w) = 1/2 h^2 sum_x omega(x) sum_d a_d(x) sum_c [(D_d v_c)(x) w_c(x) - v_c(x)
    (D_d w_c)(x)] with periodic central differences, by loops over the grid points."""
    h = 1.0 / G
    f = lambda x, c, i, j: x[c * G * G + (i % G) * G + (j % G)]
    s = 0.0
    for i in range(G):
        for j in range(G):
            om = omega[i * G + j]
            for d in range(2):
                ad = f(a, d, i, j)
                di, dj = (1, 0) if d == 0 else (0, 1)
                for c in range(2):
                    dv = (f(v, c, i + di, j + dj) - f(v, c, i - di, j - dj)) / (2 * h)
                    dw = (f(w, c, i + di, j + dj) - f(w, c, i - di, j - dj)) / (2 * h)
                    s += om * ad * (dv * f(w, c, i, j) - f(v, c, i, j) * dw)
    return 0.5 * h * h * s


def test_tensor_equals_the_form_on_the_modes():
    """Eq. tensor: C_jlk = c(psi_j, psi_l, psi_k), against the form's definition by loops."""
    m = hf.make_hf_model(G=6, K=12, R=8, decay=0.8, q_c=2, kmax=2)
    _, V = offline.pod(m.S, m.Z, 5)
    for q in range(2):
        C = offline.tensor(V, m.terms[q])
        for (j, l, k) in [(0, 0, 1), (1, 2, 3), (4, 0, 2), (3, 3, 3), (2, 4, 0)]:
            ref = brute_form(m.G, m.omega[q], V[j], V[l], V[k])
            assert abs(C[j, l, k] - ref) <= 1e-12 * max(1.0, np.abs(C).max()), (q, j, l, k)


def test_tensor_is_skew_and_multilinear(model):
    """The skew-symmetrised form gives C[j][l][k] = -C[j][k][l]; contracting the tensor with
    coefficient vectors gives the form at the reconstructed fields."""
    _, V = offline.pod(model.S, model.Z, 9)
    g = np.random.default_rng(3)
    for q in range(2):
        C = offline.tensor(V, model.terms[q])
        scale = np.abs(C).max()
        np.testing.assert_allclose(C, -C.transpose(0, 2, 1), atol=1e-13 * scale)
        a, b, c = g.standard_normal((3, 9))
        lhs = np.einsum("jlk,j,l,k->", C, a, b, c)
        rhs = offline.form(model.terms[q], a @ V, b @ V, c @ V)
        assert abs(lhs - rhs) <= 1e-12 * scale * 100


def test_form_vanishes_on_equal_last_arguments(model):
    """c(a, v, v) = 0 for the skew-symmetrised form, by the loop evaluation (pins the terms the
    synthetic model hands to the oracle and the library)."""
    g = np.random.default_rng(5)
    m = hf.make_hf_model(G=5, K=6, R=4, decay=0.8, q_c=2, kmax=2)
    a, v = g.standard_normal((2, m.N))
    for q in range(2):
        assert abs(brute_form(m.G, m.omega[q], a, v, v)) <= 1e-12
        assert abs(offline.form(m.terms[q], a, v, v)) <= 1e-12
        w = g.standard_normal(m.N)
        assert abs(offline.form(m.terms[q], a, v, w) - brute_form(m.G, m.omega[q], a, v, w)) <= 1e-11
