"""Thin ctypes binding of librb (include/rb.h): argument marshalling only.

Every function keeps the C name. Arrays are numpy (host) or torch CUDA tensors (device);
every step of the solve runs in the CUDA library. Importing this module never falls back to
another implementation: if librb.so is missing it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librb.so")

RB_OK, RB_PENDING = 0, 1
RB_ERR_ARG, RB_ERR_OOM, RB_ERR_CUDA, RB_ERR_STATE, RB_ERR_TIMEOUT = -1, -2, -3, -4, -5
RB_Q_OK, RB_Q_NOT_CONVERGED, RB_Q_SINGULAR, RB_Q_NONFINITE, RB_Q_REJECTED = 0, 1, 2, 3, 4
RB_F64, RB_F32, RB_BF16 = 0, 1, 2
RB_PREC_FP64, RB_PREC_MIXED = 0, 1
RB_THETA_TRIG, RB_THETA_USER, RB_THETA_POLY = 0, 1, 2
RB_PRESSURE_RECOVER, RB_PRESSURE_RECONSTRUCT = 0, 1
RB_N_MAX, RB_M_MAX, RB_Q_MAX = 320, 128, 64
RB_STATIC_N_MAX, RB_STATIC_SCRATCH_BYTES = 512, 16 << 20

EXPORTS = ["rb_config_default", "rb_create", "rb_destroy", "rb_last_error", "rb_load_operators",
           "rb_solve", "rb_solve_theta", "rb_solve_device", "rb_solve_device_sized",
           "rb_solve_device_status", "rb_eval", "rb_gepp_solve",
           "rb_gepp_solve_static", "rb_profile", "rb_profile_read", "rb_profile_issued", "rb_serve_start", "rb_serve_stop",
           "rb_serve_submit", "rb_serve_poll", "rb_serve_stats", "rb_serve_slots", "rb_tuning",
           "rb_load_pressure_modes", "rb_reconstruct_pressure", "rb_reconstruct_pressure_device",
           "rb_save_operators", "rb_load_operator_file", "rb_offline_pod", "rb_offline_project",
           "rb_offline_project_vector", "rb_offline_tensor"]
RB_K_NAMES = ["k_newton_fp64", "k_pressure", "k_build_x", "k_tc_gemm<plain>",
              "k_tc_gemm<sliced>", "k_lu_mixed", "k_mixed_init", "k_tc_gemm<sliced,pressure>",
              "k_newton_system", "k_prep", "k_reconstruct", "k_newton_small", "k_offline_eig",
              "k_offline_tensor"]


class rb_operators(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int), ("m", ctypes.c_int), ("q_a", ctypes.c_int),
                ("q_c", ctypes.c_int), ("q_f", ctypes.c_int), ("q_b", ctypes.c_int),
                ("dtype_c", ctypes.c_int),
                ("A", ctypes.c_void_p), ("C", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("As", ctypes.c_void_p), ("Cs", ctypes.c_void_p),
                ("fs", ctypes.c_void_p)]


class rb_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol_update", ctypes.c_double),
                ("tol_res", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("mem_budget", ctypes.c_size_t), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("theta_family", ctypes.c_int),
                ("serve_slots", ctypes.c_int), ("pressure_method", ctypes.c_int)]


class rb_csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int), ("cols", ctypes.c_int), ("indptr", ctypes.c_void_p),
                ("indices", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class rb_trilinear_term(ctypes.Structure):
    _fields_ = [("P", rb_csr), ("Q", rb_csr), ("R", rb_csr), ("weight", ctypes.c_void_p)]


RB_POD_K_MAX = 128


def _csr(M, keep):
    """rb_csr over a scipy-style CSR matrix (indptr, indices, data kept alive in `keep`)."""
    indptr = np.ascontiguousarray(M.indptr, dtype=np.int32)
    indices = np.ascontiguousarray(M.indices, dtype=np.int32)
    values = np.ascontiguousarray(M.data, dtype=np.float64)
    keep += [indptr, indices, values]
    return rb_csr(M.shape[0], M.shape[1], indptr.ctypes.data, indices.ctypes.data,
                  values.ctypes.data)


class rb_query_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("precision_used", ctypes.c_int), ("reserved", ctypes.c_int),
                ("res_norm", ctypes.c_double), ("upd_norm", ctypes.c_double)]


INFO_DTYPE = np.dtype([("status", np.int32), ("iters", np.int32), ("precision_used", np.int32),
                       ("reserved", np.int32), ("res_norm", np.float64), ("upd_norm", np.float64)])

_lib = None


def library():
    """Load librb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librb.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.rb_config_default.argtypes = [P]
        L.rb_config_default.restype = None
        L.rb_create.argtypes = [P, P, I]
        L.rb_destroy.argtypes = [P]
        L.rb_destroy.restype = None
        L.rb_last_error.argtypes = [P]
        L.rb_last_error.restype = ctypes.c_char_p
        L.rb_load_operators.argtypes = [P, P]
        L.rb_solve.argtypes = [P, P, I, P, P, P, P]
        L.rb_solve_theta.argtypes = [P, P, I, P, P, P, P]
        L.rb_solve_device.argtypes = [P, P, I, P, P, P, P, P]
        L.rb_solve_device_sized.argtypes = [P, P, I, P, P, P, P, P, P]
        L.rb_solve_device_status.argtypes = [P, I]
        L.rb_eval.argtypes = [P, P, I, I, P, I, P, P]
        L.rb_load_pressure_modes.argtypes = [P, P, I]
        L.rb_save_operators.argtypes = [P, ctypes.c_char_p]
        L.rb_load_operator_file.argtypes = [P, ctypes.c_char_p]
        L.rb_reconstruct_pressure.argtypes = [P, P, I, P, P]
        L.rb_reconstruct_pressure_device.argtypes = [P, P, I, P, P, P]
        L.rb_gepp_solve.argtypes = [P, I, I, P, P, P, P]
        L.rb_gepp_solve_static.argtypes = [I, I, P, P, P, P, P]
        L.rb_profile.argtypes = [P, I]
        L.rb_profile_read.argtypes = [P, I, P, P]
        L.rb_profile_issued.argtypes = [P, I, P]
        L.rb_serve_start.argtypes = [P]
        L.rb_serve_stop.argtypes = [P, I]
        L.rb_serve_submit.argtypes = [P, P, I, ctypes.POINTER(ctypes.c_uint64)]
        L.rb_serve_poll.argtypes = [P, ctypes.c_uint64, P, P, P]
        L.rb_serve_stats.argtypes = [P, P, P, P]
        L.rb_serve_slots.argtypes = [P]
        L.rb_tuning.argtypes = [P, I, P, P]
        L.rb_offline_pod.argtypes = [P, P, I, I, P, I, P, P]
        L.rb_offline_project.argtypes = [P, P, I, I, P, P]
        L.rb_offline_project_vector.argtypes = [P, P, I, I, P, P]
        L.rb_offline_tensor.argtypes = [P, P, I, I, P, I, P]
        for name in EXPORTS:
            if name not in ("rb_config_default", "rb_destroy", "rb_last_error"):
                getattr(L, name).restype = I
        _lib = L
    return _lib


class RbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"librb error {code}: {msg}")
        self.code = code


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def rb_gepp_solve_static(n, batch, d_M, d_rhs, d_x, d_status, stream=None):
    """No-allocation batched solve on caller-owned device buffers (torch tensors or ints)."""
    return library().rb_gepp_solve_static(n, batch, _ptr(d_M), _ptr(d_rhs), _ptr(d_x),
                                          _ptr(d_status), stream)


def rb_last_error_global() -> str:
    """Last error of a context-free call on this thread."""
    return library().rb_last_error(None).decode()


def _operators(A, C, f, B=None, As=None, Cs=None, fs=None):
    """rb_operators over host arrays (kept alive by the returned list)."""
    A, f = _f64(A), _f64(f)
    C = np.ascontiguousarray(C)
    dt = {np.dtype(np.float32): RB_F32, np.dtype(np.uint16): RB_BF16}.get(C.dtype, RB_F64)
    if dt == RB_F64:
        C = _f64(C)
    q_a, n, _ = A.shape
    ops = rb_operators(n_max=n, q_a=q_a, q_c=C.shape[0], q_f=f.shape[0], dtype_c=dt,
                       A=_ptr(A), C=_ptr(C), f=_ptr(f))
    keep = [A, C, f]
    if B is not None:
        B, As, fs = _f64(B), _f64(As), _f64(fs)
        Cs = np.ascontiguousarray(Cs, dtype=C.dtype)
        ops.m, ops.q_b = B.shape[1], B.shape[0]
        ops.B, ops.As, ops.Cs, ops.fs = _ptr(B), _ptr(As), _ptr(Cs), _ptr(fs)
        keep += [B, As, Cs, fs]
    return ops, keep


def bf16_bits(x):
    """BF16 storage of an array whose values are all BF16 numbers (float32 or float64 holding
    them): the upper 16 bits of each binary32, as uint16. Raises if a value is not a BF16
    number (no rounding happens here)."""
    x = np.asarray(x)
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    if x.dtype != np.float32 and not np.array_equal(x32.astype(x.dtype), x):
        raise ValueError("values are not BF16 numbers")
    bits = x32.view(np.uint32)
    if np.any(bits & 0xFFFF):
        raise ValueError("values are not BF16 numbers")
    return (bits >> 16).astype(np.uint16)


def _c_storage(ops, C):
    """C (or Cs) as the operator set stores it: BF16 bits for a BF16 workload."""
    if C is not None and getattr(getattr(ops, "wl", None), "c_dtype", None) == "bf16":
        return bf16_bits(C)
    return C


def rb_save_operators(path, A, C, f, B=None, As=None, Cs=None, fs=None):
    """Write an operator file (host arrays as for rb_load_operators)."""
    ops, keep = _operators(A, C, f, B, As, Cs, fs)
    rc = library().rb_save_operators(ctypes.byref(ops), os.fsencode(path))
    if rc != RB_OK:
        raise RbError(rc, f"rb_save_operators: {rb_last_error_global()}")


def save_set(path, ops):
    """Write a synth.OperatorSet (or any object with the same fields) to an operator file."""
    rb_save_operators(path, ops.A, _c_storage(ops, ops.C), ops.f, ops.B, ops.As,
                      _c_storage(ops, ops.Cs), ops.fs)


def rb_config_default() -> rb_config:
    c = rb_config()
    library().rb_config_default(ctypes.byref(c))
    return c


class Context:
    """An rb_ctx on one device. Methods mirror the C entry points one to one."""

    def __init__(self, precision=RB_PREC_FP64, tol_update=None, tol_res=None, max_iter=None,
                 mem_budget=None, use_graph=None, device=0, serve_slots=None, autotune=None,
                 theta_family=None, pressure_method=None):
        L = library()
        cfg = rb_config_default()
        cfg.precision = precision
        if tol_update is not None:
            cfg.tol_update = tol_update
        if tol_res is not None:
            cfg.tol_res = tol_res
        if max_iter is not None:
            cfg.max_iter = max_iter
        if mem_budget is not None:
            cfg.mem_budget = mem_budget
        if use_graph is not None:
            cfg.use_graph = use_graph
        if serve_slots is not None:
            cfg.serve_slots = serve_slots
        if autotune is not None:
            cfg.autotune = autotune
        if theta_family is not None:
            cfg.theta_family = theta_family
        if pressure_method is not None:
            cfg.pressure_method = pressure_method
        self.cfg = cfg
        h = ctypes.c_void_p()
        rc = L.rb_create(ctypes.byref(h), ctypes.byref(cfg), device)
        if rc != RB_OK:
            raise RbError(rc, "rb_create failed")
        self.h = h
        self.n_max = self.m = self.m_r = 0
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            library().rb_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self) -> str:
        return library().rb_last_error(self.h).decode()

    def _check(self, rc, what):
        if rc not in (RB_OK, RB_PENDING):
            raise RbError(rc, f"{what}: {self.last_error()}")
        return rc

    # --- operators ----------------------------------------------------------------------
    def rb_load_operators(self, A, C, f, B=None, As=None, Cs=None, fs=None):
        ops, keep = _operators(A, C, f, B, As, Cs, fs)
        self._check(library().rb_load_operators(self.h, ctypes.byref(ops)), "rb_load_operators")
        self.n_max, self.m = ops.n_max, (ops.m if B is not None else 0)
        self.m_r = 0
        self.q = (ops.q_a, ops.q_c, ops.q_f, ops.q_b)

    def rb_load_operator_file(self, path):
        self._check(library().rb_load_operator_file(self.h, os.fsencode(path)),
                    "rb_load_operator_file")
        with open(path, "rb") as fh:  # sizes for the output buffers, from the file's header
            h = np.frombuffer(fh.read(64), dtype="<i4")
        n, m, q_a, q_c, q_f, q_b = (int(v) for v in h[4:10])
        pres = int(h[11]) & 1
        self.n_max, self.m = n, (m if pres else 0)
        self.m_r = 0
        self.q = (q_a, q_c, q_f, q_b if pres else 0)

    def rb_load_pressure_modes(self, P_hat):
        """P_hat [m_r][n_max]: column j = pressure data of velocity basis function j."""
        P_hat = _f64(P_hat)
        self._check(library().rb_load_pressure_modes(self.h, _ptr(P_hat), P_hat.shape[0]),
                    "rb_load_pressure_modes")
        self.m_r = P_hat.shape[0]

    def rb_reconstruct_pressure(self, u, n=None):
        u = _f64(u).reshape(-1, self.n_max)
        nq = u.shape[0]
        nn = None if n is None else np.ascontiguousarray(n, dtype=np.int32)
        p = np.empty((nq, self.m_r))
        self._check(library().rb_reconstruct_pressure(self.h, _ptr(u), nq, _ptr(nn), _ptr(p)),
                    "rb_reconstruct_pressure")
        return p

    def rb_reconstruct_pressure_device(self, d_u, n_queries, d_n, d_p, stream):
        return self._check(library().rb_reconstruct_pressure_device(
            self.h, _ptr(d_u), n_queries, _ptr(d_n), _ptr(d_p), stream),
            "rb_reconstruct_pressure_device")

    def _p_out(self, nq, pressure):
        # in reconstruction mode a buffer always goes down, so that missing modes are an error
        recon = self.cfg.pressure_method == RB_PRESSURE_RECONSTRUCT
        if not pressure or (self.p_width == 0 and not recon):
            return None
        return np.empty((nq, max(self.p_width, 1)))

    @property
    def p_width(self):
        """Columns of p_out of the solves (m, or m_r when reconstructing)."""
        return self.m_r if self.cfg.pressure_method == RB_PRESSURE_RECONSTRUCT else self.m

    def load_set(self, ops):
        """Load a synth.OperatorSet (or any object with the same fields). A set that names its
        parameter-function family (wl.theta_family) must match the context's."""
        fam = getattr(getattr(ops, "wl", None), "theta_family", None)
        mine = RB_THETA_TRIG if self.cfg.theta_family == RB_THETA_USER else self.cfg.theta_family
        if fam is not None and fam != mine:
            raise ValueError(f"operator set uses theta family {fam}, the context {mine}")
        self.rb_load_operators(ops.A, _c_storage(ops, ops.C), ops.f, ops.B, ops.As,
                               _c_storage(ops, ops.Cs), ops.fs)

    # --- solves -------------------------------------------------------------------------
    def rb_solve(self, mu, n=None, pressure=True):
        mu = _f64(mu).reshape(-1, 2)
        nq = mu.shape[0]
        nn = None if n is None else np.ascontiguousarray(n, dtype=np.int32)
        u = np.empty((nq, self.n_max))
        p = self._p_out(nq, pressure)
        info = np.zeros(nq, dtype=INFO_DTYPE)
        self._check(library().rb_solve(self.h, _ptr(mu), nq, _ptr(nn), _ptr(u), _ptr(p),
                                       _ptr(info)), "rb_solve")
        return u, p, info

    def rb_solve_theta(self, theta, n=None, pressure=True):
        theta = _f64(theta)
        nq = theta.shape[0]
        nn = None if n is None else np.ascontiguousarray(n, dtype=np.int32)
        u = np.empty((nq, self.n_max))
        p = self._p_out(nq, pressure)
        info = np.zeros(nq, dtype=INFO_DTYPE)
        self._check(library().rb_solve_theta(self.h, _ptr(theta), nq, _ptr(nn), _ptr(u),
                                             _ptr(p), _ptr(info)), "rb_solve_theta")
        return u, p, info

    def rb_solve_device(self, d_mu, n_queries, d_n, d_u, d_p, d_info, stream):
        """Device pointers (torch tensors or ints) and a cudaStream_t handle (int)."""
        return self._check(library().rb_solve_device(
            self.h, _ptr(d_mu), n_queries, _ptr(d_n), _ptr(d_u), _ptr(d_p), _ptr(d_info),
            stream), "rb_solve_device")

    def rb_solve_device_sized(self, d_mu, n_queries, d_n, h_n, d_u, d_p, d_info, stream):
        """rb_solve_device with the sizes also on the host (h_n: int32 numpy array)."""
        hn = None if h_n is None else np.ascontiguousarray(h_n, dtype=np.int32)
        return self._check(library().rb_solve_device_sized(
            self.h, _ptr(d_mu), n_queries, _ptr(d_n), _ptr(hn), _ptr(d_u), _ptr(d_p),
            _ptr(d_info), stream), "rb_solve_device_sized")

    def rb_solve_device_status(self, wait=True):
        """RB_OK or RB_PENDING (wait=False); raises RbError on RB_ERR_TIMEOUT."""
        rc = library().rb_solve_device_status(self.h, 1 if wait else 0)
        if rc == RB_PENDING:
            return rc
        return self._check(rc, "rb_solve_device_status")

    # --- offline stage ------------------------------------------------------------------
    def rb_offline_pod(self, S, Z, n):
        """Modes V [n][N] (rows, orthonormal in Z) and eigenvalues [K] of the snapshots S [K][N]."""
        S = _f64(S)
        K, N = S.shape
        keep = []
        z = _csr(Z, keep)
        V = np.empty((n, N))
        lam = np.empty(K)
        self._check(library().rb_offline_pod(self.h, _ptr(S), K, N, ctypes.byref(z), n, _ptr(V),
                                             _ptr(lam)), "rb_offline_pod")
        return lam, V

    def rb_offline_project(self, V, M):
        V = _f64(V)
        n, N = V.shape
        keep = []
        m = _csr(M, keep)
        out = np.empty((n, n))
        self._check(library().rb_offline_project(self.h, _ptr(V), n, N, ctypes.byref(m), _ptr(out)),
                    "rb_offline_project")
        return out

    def rb_offline_project_vector(self, V, f):
        V, f = _f64(V), _f64(f)
        n, N = V.shape
        out = np.empty(n)
        self._check(library().rb_offline_project_vector(self.h, _ptr(V), n, N, _ptr(f), _ptr(out)),
                    "rb_offline_project_vector")
        return out

    def rb_offline_tensor(self, V, terms):
        """C [n][n][n] (index [j][l][k]) of the form given by terms [(P, Q, R, weight or None)]."""
        V = _f64(V)
        n, N = V.shape
        keep = []
        arr = (rb_trilinear_term * len(terms))()
        for i, (Pm, Qm, Rm, w) in enumerate(terms):
            wt = None if w is None else _f64(w)
            keep.append(wt)
            arr[i] = rb_trilinear_term(_csr(Pm, keep), _csr(Qm, keep), _csr(Rm, keep),
                                       None if wt is None else wt.ctypes.data)
        out = np.empty((n, n, n))
        self._check(library().rb_offline_tensor(self.h, _ptr(V), n, N, arr, len(terms), _ptr(out)),
                    "rb_offline_tensor")
        return out

    def rb_eval(self, mu, n, u, precision=RB_PREC_FP64, jacobian=True):
        mu = _f64(mu).reshape(-1, 2)
        u = _f64(u)
        nq = mu.shape[0]
        R = np.empty((nq, n))
        J = np.empty((nq, n, n)) if jacobian else None
        self._check(library().rb_eval(self.h, _ptr(mu), nq, n, _ptr(u), precision, _ptr(R),
                                      _ptr(J)), "rb_eval")
        return R, J

    def rb_gepp_solve(self, M, rhs):
        M, rhs = _f64(M), _f64(rhs)
        batch, n, _ = M.shape
        x = np.empty((batch, n))
        st = np.empty(batch, dtype=np.int32)
        self._check(library().rb_gepp_solve(self.h, n, batch, _ptr(M), _ptr(rhs), _ptr(x),
                                            _ptr(st)), "rb_gepp_solve")
        return x, st

    # --- profiling ----------------------------------------------------------------------
    def rb_profile(self, enable=True):
        return self._check(library().rb_profile(self.h, int(enable)), "rb_profile")

    def rb_profile_read(self):
        """{kernel name: (total ms, launches)} of the calls made since rb_profile(1)."""
        out = {}
        for k, name in enumerate(RB_K_NAMES):
            ms, n = ctypes.c_double(), ctypes.c_longlong()
            self._check(library().rb_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)),
                        "rb_profile_read")
            out[name] = (ms.value, n.value)
        return out

    def rb_profile_issued(self):
        """{kernel name: tensor FLOPs issued} of the GEMM kinds since rb_profile(1)."""
        out = {}
        for k in (3, 4, 7):  # RB_K_GEMM_JAC, RB_K_GEMM_RES, RB_K_GEMM_PRES
            f = ctypes.c_double()
            self._check(library().rb_profile_issued(self.h, k, ctypes.byref(f)), "rb_profile_issued")
            out[RB_K_NAMES[k]] = f.value
        return out

    # --- autotuner ----------------------------------------------------------------------
    ELIMINATION = {1: "warp per query", 2: "blocked, 32-column panels", 3: "blocked, 16-column panels",
                   4: "CTA per query, row per thread"}

    def rb_tuning(self):
        """Autotuned launch variants of every tuned size bucket (list of dicts)."""
        L = library()
        count = L.rb_tuning(self.h, -1, None, None)
        if count < 0:
            raise RbError(count, f"rb_tuning: {self.last_error()}")
        out = []
        for i in range(count):
            v = (ctypes.c_int * 6)()
            ms = (ctypes.c_float * 3)()
            L.rb_tuning(self.h, i, v, ms)
            out.append({"n_bucket": v[0], "batch_class": v[1],
                        "elimination": self.ELIMINATION.get(v[2], str(v[2])),
                        "jacobian_gemm_stages": v[3], "sliced_gemm_stages": v[4],
                        "jacobian_gemm_cta_pairs": bool(v[5] & 1),
                        "sliced_gemm_cta_pairs": bool(v[5] & 2),
                        "sliced_gemm_wide": bool(v[5] & 4),
                        "best_ms": {"elimination": ms[0], "jacobian_gemm": ms[1], "sliced_gemm": ms[2]}})
        return out

    # --- serving ------------------------------------------------------------------------
    def rb_serve_start(self):
        return self._check(library().rb_serve_start(self.h), "rb_serve_start")

    def rb_serve_stop(self, drain=True):
        return self._check(library().rb_serve_stop(self.h, int(drain)), "rb_serve_stop")

    def rb_serve_submit(self, mu, n=0):
        t = ctypes.c_uint64()
        mu = _f64(mu).reshape(2)
        self._check(library().rb_serve_submit(self.h, _ptr(mu), int(n), ctypes.byref(t)),
                    "rb_serve_submit")
        return t.value

    def rb_serve_poll(self, ticket):
        u = np.empty(self.n_max)
        p = np.empty(self.m) if self.m > 0 else None
        info = np.zeros(1, dtype=INFO_DTYPE)
        rc = self._check(library().rb_serve_poll(self.h, ticket, _ptr(u), _ptr(p), _ptr(info)),
                         "rb_serve_poll")
        if rc == RB_PENDING:
            return None
        return u, p, info[0]

    def rb_serve_slots(self):
        rc = library().rb_serve_slots(self.h)
        if rc < 0:
            raise RbError(rc, f"rb_serve_slots: {self.last_error()}")
        return rc

    def rb_serve_stats(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(library().rb_serve_stats(self.h, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(c)), "rb_serve_stats")
        return a.value, b.value, c.value
