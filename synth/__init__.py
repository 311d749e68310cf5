"""Seeded synthetic reduced operators and parameter queries.

The paper's reduced operators come from POD of high-fidelity airfoil snapshots (Sec. 3.2-3.6,
Sec. 6), which do not exist here. This module draws stand-ins with the same shapes and the
structure the paper relies on:

* affine viscous matrices A_q, q = 0..Q_a-1 (Sec. 2.4, Eq. split-a): A_0 is SPD with
  condition number about 1e3 (random orthogonal U, geometric spectrum, plus 1e-2 I);
  A_q for q >= 1 are smaller SPD corrections, sum_q>=1 ||A_q||_2 = lambda_min(A_0) / 2,
  mirroring a leading term plus small geometric corrections (Sec. 5.1);
* trilinear convection tensors C_q[j][l][k] (Sec. 3.6, Eq. tensor; j advecting, l advected,
  k test), entries N(0, 0.1^2), antisymmetrised in (l, k) as (C - C^T(l,k)) / sqrt(2) -- the
  discrete form of c(u, v, w) = -c(u, w, v) for solenoidal u;
* forcing vectors f_q ~ N(0, 1);
* pressure-recovery operators (Sec. 2.2, Eq. sup-vvar; Sec. 4.1, Eq. blocksolve-2):
  B_q (supremizer test x pressure trial; B_0 nonsymmetric, singular values in [1, 10],
  B_q>=1 small), As_q, Cs_q[j][l][k'] and fs_q;
* queries mu = (alpha in degrees, Re): alpha ~ U[0, 35], log10 Re ~ U[2, 3];
* reduced sizes per query (nested truncations of one n_max operator set);
* for the polynomial parameter family (theta_family = 2: monomials phi^q of the rotation
  angle, Sec. 5, Eq. rotsum) the q-th term of every operator is further scaled by 1/q!,
  the factor of the q-th term of the truncated rotation series R = sum_i phi^i P^i / i!.

Where a workload stores C in BF16 or FP32, the tensor is rounded here (round to nearest even)
and the rounded values *are* the operator: every solver, exact or not, sees the same numbers.

A global power-of-two scale s_A multiplies every A_q so that the problem sits in
the small-data regime where the steady solution is unique and Newton from u = 0 converges.
The bound used needs no parameter-function evaluation: |trig_q| <= 1 (and |phi^q| <= 1 for
|phi| <= 1 rad, which the polynomial workloads' angle range keeps) and
theta^a_q = theta_q / Re with Re <= Re_max give
lambda_min(A(mu)) >= s_A * lambda_min(A_0) / (2 Re_max).

This module holds random draws and data conditioning only. It evaluates no parameter
function, residual, Jacobian or solve: those belong to the method, which the oracle and the
CUDA library each implement on their own.

Seeds: PCG64 with seed = 1807_11866 + 1000 * workload id + stream id
(operators 0, queries 1, manufactured u*/p* 2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 1807_11866
STREAM_OPS, STREAM_QUERIES, STREAM_MANUFACTURED = 0, 1, 2


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes and distributions of one synthetic workload."""
    name: str
    wid: int                    # workload id, enters the seed
    n_max: int                  # reduced velocity size of the operator set
    q_a: int
    q_c: int
    q_f: int
    q_b: int = 0                # pressure affine terms (0: no pressure recovery)
    m: int = 0                  # pressure / supremizer reduced size
    batch: int = 1              # queries per solve call
    sizes: Optional[tuple] = None   # allowed reduced sizes (None: all n_max)
    size_range: Optional[tuple] = None  # (lo, hi) inclusive uniform sizes
    c_dtype: str = "f64"        # storage of C and Cs: "f64" | "f32" | "bf16"
    alpha_range: tuple = (0.0, 35.0)
    re_range: tuple = (100.0, 1000.0)
    mu0: Optional[tuple] = None     # single fixed query (manufactured workloads)
    manufactured: bool = False
    theta_family: int = 0           # 0: trigonometric functions, 2: monomials of the angle


WORKLOADS = {
    # plain single query, FP64, manufactured solution at mu0 = (10 deg, Re 200)
    "single_n20": Workload("single_n20", 0, n_max=20, q_a=4, q_c=4, q_f=2, batch=1,
                           mu0=(10.0, 200.0), re_range=(200.0, 200.0), manufactured=True),
    # parameter sweep in one launch, n = 50, pressure recovery with M = 30
    "sweep_n50": Workload("sweep_n50", 1, n_max=50, q_a=6, q_c=6, q_f=3, q_b=6, m=30,
                          batch=4096),
    # uneven batch of nested truncations of one n = 120 set, C BF16-exact
    "uneven_n120": Workload("uneven_n120", 2, n_max=120, q_a=8, q_c=8, q_f=3, batch=8192,
                            sizes=(20, 40, 80, 120), c_dtype="bf16"),
    # serving: n ~ U[16, 160], Q = 16, C FP32-exact
    "serve_n160": Workload("serve_n160", 3, n_max=160, q_a=16, q_c=16, q_f=4, batch=4096,
                           size_range=(16, 160), c_dtype="f32"),
    # large dense regime: n = 300, Q = 24, B = 16384, C BF16-exact
    "dense_n300": Workload("dense_n300", 4, n_max=300, q_a=24, q_c=24, q_f=3, batch=16384,
                           c_dtype="bf16"),
    # rotation of the airfoil by a truncated series of 12 terms (Sec. 5): polynomial parameter
    # functions with 4 * 12 + 2 viscous, 4 * 12 + 1 convective and 4 * 12 + 2 forcing terms
    "rotation_n50": Workload("rotation_n50", 5, n_max=50, q_a=50, q_c=49, q_f=50, q_b=48,
                             m=30, batch=4096, theta_family=2),
}


def rng(wid: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * wid + stream))


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even); returns float32 holding exact values."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32)


def store(x: np.ndarray, c_dtype: str) -> np.ndarray:
    if c_dtype == "f64":
        return np.ascontiguousarray(x, dtype=np.float64)
    if c_dtype == "f32":
        return np.ascontiguousarray(x, dtype=np.float32)
    if c_dtype == "bf16":
        return round_bf16(x)
    raise ValueError(c_dtype)


def haar_orthogonal(g: np.random.Generator, n: int) -> np.ndarray:
    z = g.standard_normal((n, n))
    qm, r = np.linalg.qr(z)
    return qm * np.sign(np.diag(r))[None, :]


def spd(g: np.random.Generator, n: int, lam: np.ndarray, shift: float) -> np.ndarray:
    """U diag(lam) U^T + shift I with Haar U; exactly symmetric."""
    u = haar_orthogonal(g, n)
    a = (u * lam[None, :]) @ u.T + shift * np.eye(n)
    return 0.5 * (a + a.T)


def skew_tensor(g: np.random.Generator, n: int, sigma: float = 0.1,
                out_last: Optional[int] = None) -> np.ndarray:
    """Gaussian C[j][l][k], antisymmetrised in (l, k); shape n x n x n."""
    c = g.standard_normal((n, n, n)) * sigma
    return (c - c.transpose(0, 2, 1)) / math.sqrt(2.0)


@dataclasses.dataclass
class OperatorSet:
    """Reduced affine operators for one n_max (host arrays, C-contiguous).

    A:  [q_a][n][n]  float64, row = test index k, column = trial index j
    C:  [q_c][n][n][n] (f64 or f32 storage), index [j][l][k]
    f:  [q_f][n]     float64
    B:  [q_b][m][m]  float64, row = supremizer test k', column = pressure trial i
    As: [q_a][m][n]  float64
    Cs: [q_c][n][n][m] (C storage), index [j][l][k']
    fs: [q_f][m]     float64
    """
    wl: Workload
    A: np.ndarray
    C: np.ndarray
    f: np.ndarray
    B: Optional[np.ndarray]
    As: Optional[np.ndarray]
    Cs: Optional[np.ndarray]
    fs: Optional[np.ndarray]
    s_A: float
    u_star: Optional[np.ndarray] = None
    p_star: Optional[np.ndarray] = None

    @property
    def n_max(self):
        return self.wl.n_max

    @property
    def m(self):
        return self.wl.m if self.B is not None else 0


def _frob_c(c: np.ndarray) -> float:
    return float(np.sqrt(np.sum(np.square(c, dtype=np.float64))))


def make_operators(wl: Workload, n_max: Optional[int] = None, c_dtype: Optional[str] = None,
                   q_a: Optional[int] = None, q_c: Optional[int] = None,
                   q_f: Optional[int] = None) -> OperatorSet:
    """Draw the operator set of a workload (sizes may be overridden for small test cases)."""
    wl = dataclasses.replace(
        wl,
        n_max=n_max if n_max is not None else wl.n_max,
        c_dtype=c_dtype if c_dtype is not None else wl.c_dtype,
        q_a=q_a if q_a is not None else wl.q_a,
        q_c=q_c if q_c is not None else wl.q_c,
        q_f=q_f if q_f is not None else wl.q_f,
    )
    n, g = wl.n_max, rng(wl.wid, STREAM_OPS)
    if wl.theta_family == 2 and max(abs(a) for a in wl.alpha_range) > 180.0 / math.pi:
        raise ValueError("polynomial workloads keep |alpha| <= 1 rad")

    # A_0: lambda geometric in [1e-5, 10] plus 1e-2 I -> condition ~ 1e3
    lam0 = np.geomspace(1e-5, 10.0, n) if n > 1 else np.array([10.0])
    a0 = spd(g, n, lam0, 1e-2)
    lam_min0 = float(lam0.min() + 1e-2)
    A = np.empty((wl.q_a, n, n))
    A[0] = a0
    for q in range(1, wl.q_a):
        lam = np.geomspace(1e-3, 1.0, n) if n > 1 else np.array([1.0])
        a = spd(g, n, lam, 0.0)
        A[q] = a * (lam_min0 / (2.0 * (wl.q_a - 1)))  # ||A_q||_2 = lam_min0 / (2 (Q_a - 1))

    C = np.empty((wl.q_c, n, n, n), dtype={"f64": np.float64, "f32": np.float32,
                                           "bf16": np.float32}[wl.c_dtype])
    for q in range(wl.q_c):
        C[q] = store(skew_tensor(g, n), wl.c_dtype)
    f = g.standard_normal((wl.q_f, n))

    B = As = Cs = fs = None
    if wl.q_b > 0 and wl.m > 0:
        m = wl.m
        B = np.empty((wl.q_b, m, m))
        sv = np.geomspace(1.0, 10.0, m) if m > 1 else np.array([1.0])
        B[0] = (haar_orthogonal(g, m) * sv[None, :]) @ haar_orthogonal(g, m).T
        for q in range(1, wl.q_b):
            B[q] = g.standard_normal((m, m)) * (0.5 / (wl.q_b * math.sqrt(m)))
        As = g.standard_normal((wl.q_a, m, n)) / math.sqrt(n)
        Cs = np.empty((wl.q_c, n, n, m), dtype=C.dtype)
        for q in range(wl.q_c):
            Cs[q] = store(g.standard_normal((n, n, m)) * 0.1, wl.c_dtype)
        fs = g.standard_normal((wl.q_f, m))

    if wl.theta_family == 2:
        # term q of the truncated series carries 1/q!
        def _fact(k, x):
            for q in range(1, k):
                x[q] *= 1.0 / math.factorial(q)
        _fact(wl.q_a, A)
        _fact(wl.q_c, C)
        _fact(wl.q_f, f)
        if B is not None:
            _fact(wl.q_b, B)
            _fact(wl.q_a, As)
            _fact(wl.q_c, Cs)
            _fact(wl.q_f, fs)
        if wl.c_dtype != "f64":
            for q in range(wl.q_c):
                C[q] = store(C[q], wl.c_dtype)
                if Cs is not None:
                    Cs[q] = store(Cs[q], wl.c_dtype)

    # global power-of-two scale of the viscous terms (small-data regime)
    gamma = sum(_frob_c(C[q]) for q in range(wl.q_c))
    re_max, re_min = max(wl.re_range), min(wl.re_range)
    c_lo = lam_min0 / (2.0 * re_max)  # lambda_min(A(mu)) >= s_A * c_lo
    u_star = p_star = None
    if wl.manufactured:
        gm = rng(wl.wid, STREAM_MANUFACTURED)
        u_star = gm.standard_normal(n)
        p_star = gm.standard_normal(wl.m) if B is not None else None
        # moderate nonlinearity at the manufactured root: lambda_lo >= 4 gamma ||u*||
        need = 4.0 * gamma * float(np.linalg.norm(u_star)) / c_lo
    else:
        fnorm = sum(float(np.linalg.norm(f[q])) for q in range(wl.q_f))
        # classical uniqueness: lambda_lo^2 >= 4 gamma ||f||
        need = math.sqrt(4.0 * gamma * fnorm) / c_lo
    k = max(0, math.ceil(math.log2(max(need, 1.0))))
    s_A = float(2.0 ** k)
    A *= s_A
    return OperatorSet(wl, A, C, f, B, As, Cs, fs, s_A, u_star, p_star)


@dataclasses.dataclass
class QuerySet:
    mu: np.ndarray      # [B][2] float64: alpha (degrees), Re
    n: np.ndarray       # [B] int32 reduced sizes


def make_queries(wl: Workload, batch: Optional[int] = None, n_max: Optional[int] = None) -> QuerySet:
    b = batch if batch is not None else wl.batch
    nm = n_max if n_max is not None else wl.n_max
    g = rng(wl.wid, STREAM_QUERIES)
    if wl.mu0 is not None:
        mu = np.tile(np.array(wl.mu0, dtype=np.float64), (b, 1))
    else:
        alpha = g.uniform(wl.alpha_range[0], wl.alpha_range[1], b)
        lo, hi = math.log10(wl.re_range[0]), math.log10(wl.re_range[1])
        re = 10.0 ** g.uniform(lo, hi, b)
        mu = np.stack([alpha, re], axis=1)
    if wl.sizes is not None:
        sizes = np.array([s for s in wl.sizes if s <= nm] or [nm], dtype=np.int32)
        n = g.choice(sizes, b).astype(np.int32)
    elif wl.size_range is not None:
        lo, hi = wl.size_range
        n = g.integers(min(lo, nm), min(hi, nm) + 1, b).astype(np.int32)
    else:
        n = np.full(b, nm, dtype=np.int32)
    return QuerySet(np.ascontiguousarray(mu), np.ascontiguousarray(n))


def corner_queries(wl: Workload) -> np.ndarray:
    """The four corners of the parameter box (always part of parity samples)."""
    a0, a1 = wl.alpha_range
    r0, r1 = min(wl.re_range), max(wl.re_range)
    return np.array([[a0, r0], [a0, r1], [a1, r0], [a1, r1]], dtype=np.float64)


def stratified_indices(wl: Workload, mu: np.ndarray, cells=(6, 10)) -> np.ndarray:
    """Indices of queries spread over the parameter box, for parity samples: the box is cut into
    cells[0] x cells[1] cells (alpha linear, log10 Re), and from each cell the query nearest its
    centre is taken (cells without a query are skipped). Sorted, distinct."""
    a0, a1 = wl.alpha_range
    r0, r1 = math.log10(min(wl.re_range)), math.log10(max(wl.re_range))
    na, nr = cells
    x = (mu[:, 0] - a0) / max(a1 - a0, 1e-300) * na
    y = (np.log10(mu[:, 1]) - r0) / max(r1 - r0, 1e-300) * nr
    ca = np.clip(np.floor(x), 0, na - 1).astype(int)
    cr = np.clip(np.floor(y), 0, nr - 1).astype(int)
    d = (x - ca - 0.5) ** 2 + (y - cr - 0.5) ** 2
    pick = {}
    for i in np.argsort(d, kind="stable"):
        pick.setdefault((ca[i], cr[i]), int(i))
    return np.array(sorted(pick.values()), dtype=np.int64)
