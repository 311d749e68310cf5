"""Checks of the seeded synthetic inputs (structure only; no method arithmetic)."""
import dataclasses
import math

import numpy as np
import pytest

import synth


def test_seeds_reproduce_bit_for_bit():
    wl = synth.WORKLOADS["sweep_n50"]
    a = synth.make_operators(wl, n_max=12)
    b = synth.make_operators(wl, n_max=12)
    for x, y in [(a.A, b.A), (a.C, b.C), (a.f, b.f), (a.B, b.B), (a.Cs, b.Cs)]:
        np.testing.assert_array_equal(x, y)
    qa, qb = synth.make_queries(wl, batch=64), synth.make_queries(wl, batch=64)
    np.testing.assert_array_equal(qa.mu, qb.mu)


@pytest.mark.parametrize("c_dtype", ["f64", "f32", "bf16"])
def test_skew_exact_in_storage(c_dtype):
    ops = synth.make_operators(synth.WORKLOADS["sweep_n50"], n_max=10, c_dtype=c_dtype)
    np.testing.assert_array_equal(ops.C, -ops.C.transpose(0, 1, 3, 2))


def test_bf16_rounding_exact_and_nearest():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 1e-30, 65504.0], np.float64)
    r = synth.round_bf16(x)
    bits = r.view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert r[0] == 1.0
    assert r[1] == 1.0  # tie -> even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] - x[3]) <= 2 ** -8 * abs(x[3])


def test_viscous_spectrum_and_scaling():
    ops = synth.make_operators(synth.WORKLOADS["sweep_n50"], n_max=30)
    s = ops.s_A
    ev = np.linalg.eigvalsh(ops.A[0] / s)
    assert ev.min() > 0
    assert 5e2 < ev.max() / ev.min() < 2e3
    corr = sum(np.linalg.norm(ops.A[q] / s, 2) for q in range(1, ops.A.shape[0]))
    assert corr <= 0.5 * ev.min() * (1 + 1e-9)
    assert s == 2.0 ** round(np.log2(s))


def test_nested_truncation_is_prefix():
    wl = synth.WORKLOADS["uneven_n120"]
    q = synth.make_queries(wl, batch=256)
    assert set(np.unique(q.n)) <= {20, 40, 80, 120}
    assert q.mu[:, 0].min() >= 0 and q.mu[:, 0].max() <= 35
    assert q.mu[:, 1].min() >= 100 and q.mu[:, 1].max() <= 1000


def test_pressure_operator_nonsingular():
    ops = synth.make_operators(synth.WORKLOADS["sweep_n50"], n_max=8)
    sv = np.linalg.svd(ops.B[0], compute_uv=False)
    assert sv.min() > 0.9 and sv.max() < 11


def test_rotation_workload_factorial_terms():
    # term q of every operator of the polynomial workload carries 1/q! on top of the draw
    wl = synth.WORKLOADS["rotation_n50"]
    assert wl.theta_family == 2 and (wl.q_a, wl.q_c, wl.q_f) == (50, 49, 50)
    ops = synth.make_operators(wl, n_max=6)
    for q in (1, 5, 12):
        assert np.max(np.abs(ops.f[q])) < 10.0 / math.factorial(q)
        assert np.max(np.abs(ops.C[q])) < 1.0 / math.factorial(q)
    with pytest.raises(ValueError):
        synth.make_operators(dataclasses.replace(wl, alpha_range=(0.0, 90.0)), n_max=4)
