"""The double -> double-float split and the float -> double widening that the kernels do with
integer operations (rb_internal.cuh), checked bit for bit on the GPU against the plain FP64
conversions: random values over every binade around the FP32 range, ties at the rounding point,
carries into the next binade, the range edges, zeros, subnormals, infinities and NaN."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1807_11866_gb300 import _build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("split") / "libsplit_check.so")
    cmd = [_build.nvcc(), *_build.NVCC_FLAGS, "-shared", os.path.join(HERE, "cuda", "split_check.cu"),
           "-o", out, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    lib.split_check.restype = ctypes.c_int
    lib.split_check.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                ctypes.c_void_p]
    return lib


def doubles_from(sign, exp_field, mant):
    bits = (np.asarray(sign, np.uint64) << np.uint64(63)) | (np.asarray(exp_field, np.uint64) << np.uint64(52)) \
        | np.asarray(mant, np.uint64)
    return bits.view(np.float64)


def split_inputs():
    g = np.random.default_rng(11)
    n = 1 << 18
    sign = g.integers(0, 2, n)
    e = g.integers(-80, 131, n) + 1023
    mant = g.integers(0, 1 << 52, n, dtype=np.uint64)
    v = [doubles_from(sign, e, mant)]
    # ties: the 29 bits below the FP32 significand exactly one half, top bits odd and even
    m = 3000
    top = g.integers(0, 1 << 23, m, dtype=np.uint64)
    ties = (top << np.uint64(29)) | np.uint64(1 << 28)
    ee = g.integers(-74, 127, m) + 1023
    v.append(doubles_from(g.integers(0, 2, m), ee, ties))
    # carries: all 23 top bits set, the rest at or above one half
    rest = g.integers(1 << 28, 1 << 29, m, dtype=np.uint64)
    car = (np.uint64((1 << 23) - 1) << np.uint64(29)) | rest
    v.append(doubles_from(g.integers(0, 2, m), ee, car))
    # range edges and special values
    edges = []
    for eu in (-76, -75, -74, -73, 125, 126, 127, 128):
        for mm in (0, 1, (1 << 52) - 1, (((1 << 23) - 1) << 29) | (1 << 28), 1 << 28, 3 << 28):
            for s in (0, 1):
                edges.append(doubles_from(s, eu + 1023, mm))
    edges += [np.array([0.0, -0.0, 5e-324, -5e-324, 2.2e-308, np.inf, -np.inf, np.nan, 1e300,
                        -1e300, 3.4028234663852886e38, 3.4028235677973366e38, 1.0, -1.0, 0.5,
                        1e-30, 1e-23, 2.0 ** -74, 2.0 ** -75])]
    v.append(np.concatenate([np.atleast_1d(x) for x in edges]))
    return np.ascontiguousarray(np.concatenate(v), dtype=np.float64)


def float_inputs():
    g = np.random.default_rng(12)
    bits = g.integers(0, 1 << 32, 1 << 18, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, 1e-45, -1e-45, 1.1754942e-38, 1.1754944e-38, np.inf, -np.inf,
                        np.nan, 3.4028235e38, 1.0, -2.5], dtype=np.float32)
    return np.ascontiguousarray(np.concatenate([bits.view(np.float32), special]))


def test_split_matches_fp64_conversions(checker):
    v = split_inputs()
    x = float_inputs()
    bad = (ctypes.c_int * 2)()
    rc = checker.split_check(v.ctypes.data, v.size, x.ctypes.data, x.size, bad)
    assert rc >= 0, "CUDA error in the split check"
    msg = []
    if bad[0] != 0x7FFFFFFF:
        msg.append(f"df_split differs at {v[bad[0]]!r} (bits {v[bad[0]:bad[0]+1].view(np.uint64)[0]:#018x})")
    if bad[1] != 0x7FFFFFFF:
        msg.append(f"f32_to_f64 differs at {x[bad[1]]!r}")
    assert rc == 0, "; ".join(msg)
