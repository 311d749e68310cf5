"""A seeded synthetic high-fidelity model for the offline stage (Sec. 3.2, 3.5, 3.6).

The paper's high-fidelity spaces (divergence-conforming B-splines on the NACA0015 domain) and
their snapshots are not available. This module draws stand-ins with the structure the offline
stage relies on, as sparse matrices and arrays (inputs only: it performs no step of the reduced
basis method -- no covariance, eigen-decomposition, projection or tensor reduction):

* a doubly periodic G x G grid of spacing h = 1/G carrying a velocity field with two components,
  dof index c G^2 + i G + j (component c, x-index i, y-index j): N_h = 2 G^2;
* central differences D_x, D_y (periodic, per component) and the component selections E_0, E_1
  (G^2 x N_h);
* the H1-seminorm covariance matrix Z = the 5-point stiffness (4 on the diagonal, -1 per
  neighbour, per component), the velocity covariance of Sec. 3.2 (Eq. for z_V), also the first
  viscous affine matrix; a mass matrix h^2 I as the second;
* convection forms c_q(a, v, w) = 1/2 h^2 sum_x omega_q(x) sum_{d,c} a_d(x) [(D_d v)_c(x) w_c(x)
  - v_c(x) (D_d w)_c(x)], skew in (v, w) by construction (the discrete form of c(u, v, w) =
  -c(u, w, v)), given as pointwise quadrature terms (P, Q, R, weight):
  c(a, v, w) = sum_terms sum_x weight(x) (P a)(x) (Q v)(x) (R w)(x); omega_0 = 1, omega_1 a smooth
  positive field;
* forcing vectors: smooth random fields times h^2;
* snapshots: K fields sum_m sigma_m a_im phi_m of R smooth divergence-free fields phi_m (curl of
  a random Fourier stream function: discretely divergence-free for the central differences),
  sigma_m = decay^m, a_im ~ N(0, 1): a covariance spectrum that decays geometrically.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from . import rng

HF_WID = 6  # workload id of the offline stage's seeds


@dataclasses.dataclass
class HFModel:
    G: int
    h: float
    N: int                  # N_h = 2 G^2
    Z: sp.csr_matrix        # covariance (H1 seminorm), also A_0
    A: list                 # affine viscous matrices [A_0, A_1]
    f: np.ndarray           # [q_f][N]
    terms: list             # per convection affine term: list of (P, Q, R, weight)
    S: np.ndarray           # snapshots [K][N]
    Dx: sp.csr_matrix
    Dy: sp.csr_matrix
    E: list                 # component selections [E_0, E_1]
    omega: list             # per convection term: weight field [G^2]


def _cyclic_diff(G: int, h: float) -> sp.csr_matrix:
    """1-D periodic central difference (v[i+1] - v[i-1]) / (2h)."""
    d = sp.lil_matrix((G, G))
    for i in range(G):
        d[i, (i + 1) % G] += 1.0 / (2 * h)
        d[i, (i - 1) % G] -= 1.0 / (2 * h)
    return d.tocsr()


def _cyclic_lap(G: int) -> sp.csr_matrix:
    """1-D periodic second difference pattern: 2 on the diagonal, -1 per neighbour."""
    d = sp.lil_matrix((G, G))
    for i in range(G):
        d[i, i] += 2.0
        d[i, (i + 1) % G] -= 1.0
        d[i, (i - 1) % G] -= 1.0
    return d.tocsr()


def _smooth_field(g: np.random.Generator, G: int, kmax: int, p: float) -> np.ndarray:
    """Real random Fourier field on the periodic grid, |k| <= kmax, amplitude |k|^-p, zero mean."""
    x = np.arange(G) / G
    X, Y = np.meshgrid(x, x, indexing="ij")
    out = np.zeros((G, G))
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if kx == 0 and ky == 0:
                continue
            amp = (kx * kx + ky * ky) ** (-p / 2)
            a, b = g.standard_normal(2) * amp
            ph = 2 * math.pi * (kx * X + ky * Y)
            out += a * np.cos(ph) + b * np.sin(ph)
    return out


def make_hf_model(G: int = 128, K: int = 128, R: int = 60, decay: float = 0.85, q_c: int = 2,
                  q_f: int = 2, kmax: int = 6) -> HFModel:
    g = rng(HF_WID, 0)
    h = 1.0 / G
    n2 = G * G
    N = 2 * n2
    I_G = sp.identity(G, format="csr")
    d1 = _cyclic_diff(G, h)
    l1 = _cyclic_lap(G)
    # scalar-field operators on index i G + j (i: x, j: y)
    dx_s = sp.kron(d1, I_G, format="csr")
    dy_s = sp.kron(I_G, d1, format="csr")
    lap_s = (sp.kron(l1, I_G) + sp.kron(I_G, l1)).tocsr()
    I2 = sp.identity(2, format="csr")
    Dx = sp.kron(I2, dx_s, format="csr")
    Dy = sp.kron(I2, dy_s, format="csr")
    Z = sp.kron(I2, lap_s, format="csr")
    Mass = (h * h) * sp.identity(N, format="csr")
    E = [sp.hstack([sp.identity(n2), sp.csr_matrix((n2, n2))], format="csr"),
         sp.hstack([sp.csr_matrix((n2, n2)), sp.identity(n2)], format="csr")]
    omega = [np.ones(n2)]
    for q in range(1, q_c):
        w = _smooth_field(g, G, 3, 2.0)
        omega.append((1.0 + 0.5 * w / np.abs(w).max()).reshape(-1))
    D = [Dx, Dy]
    terms = []
    for q in range(q_c):
        tq = []
        wt = 0.5 * h * h * omega[q]
        for d in range(2):
            for c in range(2):
                tq.append((E[d], (E[c] @ D[d]).tocsr(), E[c], wt.copy()))
                tq.append((E[d], E[c], (E[c] @ D[d]).tocsr(), -wt))
        terms.append(tq)
    f = np.stack([(h * h) * np.concatenate([_smooth_field(g, G, 4, 1.5).reshape(-1),
                                            _smooth_field(g, G, 4, 1.5).reshape(-1)])
                  for _ in range(q_f)])
    # divergence-free fields: u = D_y psi, v = -D_x psi for random stream functions psi
    fields = []
    for m in range(R):
        psi = _smooth_field(g, G, kmax, 2.5).reshape(-1)
        fields.append(np.concatenate([dy_s @ psi, -(dx_s @ psi)]))
    Phi = np.stack(fields)                       # [R][N]
    Phi /= np.sqrt(np.einsum("rn,rn->r", Phi, (Z @ Phi.T).T))[:, None]  # unit H1 seminorm
    sigma = decay ** np.arange(R)
    a = g.standard_normal((K, R))
    S = (a * sigma[None, :]) @ Phi               # [K][N]
    return HFModel(G, h, N, Z, [Z, Mass], f, terms, S, Dx, Dy, E, omega)


def csr_arrays(M: sp.csr_matrix):
    """(indptr, indices, values) of a CSR matrix as int32 / float64 arrays."""
    M = sp.csr_matrix(M)
    M.sort_indices()
    return (np.ascontiguousarray(M.indptr, dtype=np.int32),
            np.ascontiguousarray(M.indices, dtype=np.int32),
            np.ascontiguousarray(M.data, dtype=np.float64))
