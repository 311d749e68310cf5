"""Oracle: plain FP64 CPU restatement of the online stage (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import this
package. The product library never loads it, and it shares no code with the CUDA path.

The arithmetic lives in ``rb_oracle.c`` (plain C, no BLAS, OpenMP across queries); this
module compiles it with gcc and wraps it with ctypes. ``manufacture`` builds the forcing of a
manufactured-solution workload from the oracle's own residual.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q_OK, Q_NOT_CONVERGED, Q_SINGULAR, Q_NONFINITE = 0, 1, 2, 3


class _Ops(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int), ("m", ctypes.c_int), ("q_a", ctypes.c_int),
                ("q_c", ctypes.c_int), ("q_f", ctypes.c_int), ("q_b", ctypes.c_int),
                ("c_is_f32", ctypes.c_int),
                ("A", ctypes.c_void_p), ("C", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("As", ctypes.c_void_p), ("Cs", ctypes.c_void_p),
                ("fs", ctypes.c_void_p), ("theta_family", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("res_norm", ctypes.c_double), ("upd_norm", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile rb_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or \
                os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
                                   "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        L.oracle_theta.argtypes = [P, ctypes.c_double, ctypes.c_double, P]
        L.oracle_assemble.argtypes = [P, ctypes.c_int, P, P, P]
        L.oracle_convection.argtypes = [P, ctypes.c_int, P, P, P]
        L.oracle_residual.argtypes = [P, ctypes.c_int, P, P, P]
        L.oracle_jacobian.argtypes = [P, ctypes.c_int, P, P, P]
        L.oracle_gepp_solve.argtypes = [ctypes.c_int, P, P]
        L.oracle_gepp_solve.restype = ctypes.c_int
        L.oracle_newton_theta.argtypes = [P, ctypes.c_int, P, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, P, P, P, P]
        L.oracle_pressure_theta.argtypes = [P, ctypes.c_int, P, P, P]
        L.oracle_reconstruct.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        L.oracle_reconstruct.restype = None
        L.oracle_pressure_theta.restype = ctypes.c_int
        L.oracle_solve_batch.argtypes = [P, ctypes.c_int, P, P, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, P, P, P, ctypes.c_int]
        L.oracle_solve_theta_batch.argtypes = [P, ctypes.c_int, P, P, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int, P, P, P,
                                               ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """Holds one operator set (host arrays, kept alive) for the C oracle."""

    def __init__(self, A, C, f, B=None, As=None, Cs=None, fs=None, theta_family=0):
        self.A = np.ascontiguousarray(A, dtype=np.float64)
        c_is_f32 = np.asarray(C).dtype == np.float32
        cdt = np.float32 if c_is_f32 else np.float64
        self.C = np.ascontiguousarray(C, dtype=cdt)
        self.f = np.ascontiguousarray(f, dtype=np.float64)
        self.q_a, n, _ = self.A.shape
        self.q_c = self.C.shape[0]
        self.q_f = self.f.shape[0]
        self.n_max = n
        assert self.C.shape[1:] == (n, n, n) and self.f.shape[1] == n
        if B is not None:
            self.B = np.ascontiguousarray(B, dtype=np.float64)
            self.As = np.ascontiguousarray(As, dtype=np.float64)
            self.Cs = np.ascontiguousarray(Cs, dtype=cdt)
            self.fs = np.ascontiguousarray(fs, dtype=np.float64)
            self.q_b, self.m, _ = self.B.shape
        else:
            self.B = self.As = self.Cs = self.fs = None
            self.q_b = self.m = 0
        self._ops = _Ops(self.n_max, self.m, self.q_a, self.q_c, self.q_f, self.q_b,
                         int(c_is_f32), _ptr(self.A), _ptr(self.C), _ptr(self.f),
                         _ptr(self.B), _ptr(self.As), _ptr(self.Cs), _ptr(self.fs),
                         int(theta_family))
        self.n_theta = self.q_a + self.q_c + self.q_f + self.q_b

    @classmethod
    def from_set(cls, ops):
        return cls(ops.A, ops.C, ops.f, ops.B, ops.As, ops.Cs, ops.fs,
                   theta_family=getattr(ops.wl, "theta_family", 0))

    @property
    def ref(self):
        return ctypes.byref(self._ops)

    # --- single-query building blocks -------------------------------------------------
    def theta(self, alpha_deg, re):
        t = np.empty(self.n_theta)
        lib().oracle_theta(self.ref, float(alpha_deg), float(re), _ptr(t))
        return t

    def assemble(self, n, theta):
        A = np.empty((n, n))
        f = np.empty(n)
        lib().oracle_assemble(self.ref, n, _ptr(np.ascontiguousarray(theta, np.float64)),
                              _ptr(A), _ptr(f))
        return A, f

    def convection(self, n, theta, u):
        out = np.empty(n)
        lib().oracle_convection(self.ref, n, _ptr(np.ascontiguousarray(theta, np.float64)),
                                _ptr(np.ascontiguousarray(u, np.float64)), _ptr(out))
        return out

    def residual(self, n, theta, u):
        out = np.empty(n)
        lib().oracle_residual(self.ref, n, _ptr(np.ascontiguousarray(theta, np.float64)),
                              _ptr(np.ascontiguousarray(u, np.float64)), _ptr(out))
        return out

    def jacobian(self, n, theta, u):
        out = np.empty((n, n))
        lib().oracle_jacobian(self.ref, n, _ptr(np.ascontiguousarray(theta, np.float64)),
                              _ptr(np.ascontiguousarray(u, np.float64)), _ptr(out))
        return out

    def newton(self, n, theta, tol_upd=1e-10, tol_res=1e-10, max_iter=50):
        u = np.empty(n)
        info = Info()
        tr = np.zeros(max_iter)
        tu = np.zeros(max_iter)
        lib().oracle_newton_theta(self.ref, n, _ptr(np.ascontiguousarray(theta, np.float64)),
                                  tol_upd, tol_res, max_iter, _ptr(u), ctypes.byref(info),
                                  _ptr(tr), _ptr(tu))
        k = info.iters
        return u, info, tr[:k], tu[:k]

    def pressure(self, n, theta, u):
        p = np.empty(self.m)
        rc = lib().oracle_pressure_theta(self.ref, n,
                                         _ptr(np.ascontiguousarray(theta, np.float64)),
                                         _ptr(np.ascontiguousarray(u, np.float64)), _ptr(p))
        return p, rc

    # --- batches ------------------------------------------------------------------------
    def solve(self, mu, n=None, tol_upd=1e-10, tol_res=1e-10, max_iter=50, threads=0,
              pressure=True):
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1, 2)
        nq = mu.shape[0]
        nsz = None if n is None else np.ascontiguousarray(n, dtype=np.int32)
        u = np.empty((nq, self.n_max))
        p = np.empty((nq, self.m)) if (pressure and self.m > 0) else None
        info = (Info * max(nq, 1))()
        lib().oracle_solve_batch(self.ref, nq, _ptr(mu), _ptr(nsz), tol_upd, tol_res, max_iter,
                                 _ptr(u), _ptr(p), info, threads)
        return u, p, _info_arrays(info, nq)

    def solve_theta(self, theta, n=None, tol_upd=1e-10, tol_res=1e-10, max_iter=50,
                    threads=0, pressure=True):
        theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, self.n_theta)
        nq = theta.shape[0]
        nsz = None if n is None else np.ascontiguousarray(n, dtype=np.int32)
        u = np.empty((nq, self.n_max))
        p = np.empty((nq, self.m)) if (pressure and self.m > 0) else None
        info = (Info * max(nq, 1))()
        lib().oracle_solve_theta_batch(self.ref, nq, _ptr(theta), _ptr(nsz), tol_upd, tol_res,
                                       max_iter, _ptr(u), _ptr(p), info, threads)
        return u, p, _info_arrays(info, nq)


def reconstruct(P_hat, u, n=None):
    """Pressure reconstruction p = sum_{j < n} u_j P_hat[:, j] (Sec. 4.2), one query per row of u."""
    P_hat = np.ascontiguousarray(P_hat, dtype=np.float64)
    m_r, n_max = P_hat.shape
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, n_max)
    nn = np.full(u.shape[0], n_max, np.int32) if n is None else np.asarray(n, np.int32).reshape(-1)
    p = np.empty((u.shape[0], m_r))
    for b in range(u.shape[0]):
        lib().oracle_reconstruct(_ptr(P_hat), m_r, n_max, int(nn[b]), _ptr(u[b]), _ptr(p[b]))
    return p


def gepp_solve(M, rhs):
    """Solve M_s x_s = rhs_s for every system s of a batch by the oracle's Gaussian elimination
    with partial pivoting (first row of largest magnitude). M [batch][n][n], rhs [batch][n].
    Returns x [batch][n] (0 for a singular system) and status [batch] (0 ok, 2 singular)."""
    M = np.array(M, dtype=np.float64, copy=True, order="C")
    x = np.array(rhs, dtype=np.float64, copy=True, order="C")
    batch, n = x.shape
    st = np.zeros(batch, np.int32)
    for s in range(batch):
        if lib().oracle_gepp_solve(n, _ptr(M[s]), _ptr(x[s])):
            st[s] = Q_SINGULAR
            x[s] = 0.0
    return x, st


def _info_arrays(info, nq):
    return {
        "status": np.array([info[i].status for i in range(nq)], dtype=np.int32),
        "iters": np.array([info[i].iters for i in range(nq)], dtype=np.int32),
        "res_norm": np.array([info[i].res_norm for i in range(nq)]),
        "upd_norm": np.array([info[i].upd_norm for i in range(nq)]),
    }


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def manufacture(ops, mu0):
    """Overwrite f_0 (and fs_0) of a synthetic operator set so that u* (and p*) solve the
    problem exactly at mu0: f_0 = A(mu0) u* + Cmu0(u*, u*) - sum_{q>=1} theta^f_q f_q
    (theta^f_0 = 1), and fs_0 = B(mu0) p* + As(mu0) u* + Cs_mu0(u*, u*) - sum_{q>=1} ...
    Uses the oracle's own residual; the result is an oracle-side input for the tests."""
    o = Oracle.from_set(ops)
    n = o.n_max
    th = o.theta(*mu0)
    f = ops.f.copy()
    f[0] = 0.0
    o2 = Oracle(ops.A, ops.C, f)
    # with f_0 = 0, R(u*) = A u* + C(u*,u*) - sum_{q>=1} theta^f_q f_q
    f[0] = o2.residual(n, th[:o2.n_theta], ops.u_star) / th[o.q_a + o.q_c]
    ops.f = f
    if ops.B is not None and ops.p_star is not None:
        fs = ops.fs.copy()
        fs[0] = 0.0
        o3 = Oracle(ops.A, ops.C, f, ops.B, ops.As, ops.Cs, fs)
        th3 = o3.theta(*mu0)
        # with fs_0 = 0 the recovered right-hand side is r = -As u* - Cs(u*,u*) + ...
        # so fs_0 = B(mu0) p* - r(u*) makes B p* = r hold.
        tb = th3[o3.q_a + o3.q_c + o3.q_f:]
        Bm = np.tensordot(tb, ops.B, axes=1)
        rhs0 = _pressure_rhs(o3, n, th3, ops.u_star)
        fs[0] = (Bm @ ops.p_star - rhs0) / th3[o3.q_a + o3.q_c]
        ops.fs = fs
    return ops


def _pressure_rhs(o, n, theta, u):
    """fs(mu) - As(mu) u - Cs_mu(u, u) evaluated through the oracle's pressure routine with
    B replaced by the identity (solve of I p = r returns r)."""
    eye = np.zeros_like(o.B)
    eye[0] = np.eye(o.m)
    tb0 = theta[o.q_a + o.q_c + o.q_f]
    o_id = Oracle(o.A, o.C, o.f, eye / tb0, o.As, o.Cs, o.fs)
    p, rc = o_id.pressure(n, theta, u)
    assert rc == 0
    return p
