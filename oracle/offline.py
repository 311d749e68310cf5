"""Oracle of the offline stage (test infrastructure only): plain FP64 numpy restatement of the
reduced-basis construction the online stage starts from.

Only the test suite and the benchmark's CPU-baseline leg may import this module. It shares no
code with the CUDA path.

* POD by the method of snapshots (Sec. 3.2): the covariance matrix C_ij = z(phi_i, phi_j)
  (Eq. covmx), its eigenpairs (lambda_j, v^j) in decreasing order, and the modes
  psi_j = lambda_j^(-1/2) sum_i v^j_i phi_i (Eq. spd). The symmetric eigenproblem is solved by
  LAPACK (numpy.linalg.eigh), a library primitive.
* Galerkin projection of a high-fidelity matrix or vector onto the modes (Sec. 3.5,
  Eq. redorth-final): M^R = V^T M^H V, f^R = V^T f^H, V's columns the modes.
* The third-order tensor of a trilinear form (Sec. 3.6, Eq. tensor): C_jlk = c(psi_j, psi_l,
  psi_k) for a form given by pointwise quadrature terms,
  c(a, v, w) = sum_terms sum_x weight(x) (P a)(x) (Q v)(x) (R w)(x).
"""
from __future__ import annotations

import numpy as np


def covariance(S, Z):
    """C_ij = z(phi_i, phi_j) = phi_i^T Z phi_j for the snapshots S [K][N] (Eq. covmx)."""
    S = np.asarray(S, dtype=np.float64)
    ZS = np.asarray(Z @ S.T)            # [N][K]
    return S @ ZS


def pod(S, Z, n):
    """POD by the method of snapshots (Eqs. covmx, spd): returns (lambda [K] decreasing,
    modes V [n][N] with V Z V^T = I)."""
    S = np.asarray(S, dtype=np.float64)
    C = covariance(S, Z)
    C = 0.5 * (C + C.T)
    lam, W = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam, W = lam[order], W[:, order]
    V = (W[:, :n] / np.sqrt(lam[:n])[None, :]).T @ S      # psi_j = sum_i v^j_i phi_i / sqrt(l_j)
    return lam, V


def project(V, M):
    """M^R = V M V^T with the modes as the rows of V [n][N] (Eq. redorth-final)."""
    V = np.asarray(V, dtype=np.float64)
    return V @ np.asarray(M @ V.T)


def project_vector(V, f):
    """f^R = V f (the reduced right-hand side)."""
    return np.asarray(V, dtype=np.float64) @ np.asarray(f, dtype=np.float64)


def tensor(V, terms):
    """C[j][l][k] = sum_terms sum_x w(x) (P psi_j)(x) (Q psi_l)(x) (R psi_k)(x) (Eq. tensor);
    index j advecting, l advected, k test. terms: list of (P, Q, R, weight or None)."""
    V = np.asarray(V, dtype=np.float64)
    n = V.shape[0]
    C = np.zeros((n, n, n))
    for P, Q, R, w in terms:
        EP = np.asarray(P @ V.T)        # [points][n]
        EQ = np.asarray(Q @ V.T)
        ER = np.asarray(R @ V.T)
        if w is not None:
            EP = EP * np.asarray(w, dtype=np.float64)[:, None]
        C += np.einsum("xj,xl,xk->jlk", EP, EQ, ER, optimize=True)
    return C


def form(terms, a, v, w):
    """The high-fidelity trilinear form itself at full vectors a, v, w [N]."""
    s = 0.0
    for P, Q, R, wt in terms:
        pa, qv, rw = P @ a, Q @ v, R @ w
        s += float(np.sum((wt if wt is not None else 1.0) * pa * qv * rw))
    return s
