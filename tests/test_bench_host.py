"""Host logic of bench.py on the CPU: the algorithmic work behind the roofline figures (chord
steps counted as triangular solves) and the combined-basis construction used to compare
pressure reconstruction with recovery."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402

INFO = np.dtype([("status", np.int32), ("iters", np.int32), ("precision_used", np.int32),
                 ("reserved", np.int32), ("res_norm", np.float64), ("upd_norm", np.float64)])


def test_roofline_work_counts_chord_steps():
    wl = synth.WORKLOADS["sweep_n50"]
    q = synth.QuerySet(np.zeros((4, 2)), np.full(4, 50, np.int32))
    info = np.zeros(4, INFO)
    info["iters"] = [4, 4, 3, 2]
    kprof = {"k_lu_mixed": (1.0, 4), "k_tc_gemm<plain>": (1.0, 2), "k_newton_system": (1.0, 4),
             "k_tc_gemm<sliced>": (1.0, 2)}
    n = 50.0
    for chord in (True, False):
        issued = {"k_tc_gemm<plain>": 7.0e9, "k_tc_gemm<sliced>": 3.0e10}  # device-counted FLOPs
        _, rl, _ = bench.kernel_rooflines(1, wl, q, info, kprof, 1, np.full(4, chord), issued)
        it = np.array([4, 4, 3, 2], float)
        full = np.minimum(it, 3) if chord else it
        chs = it - full
        lu = np.sum(full * (2 * n ** 3 / 3 + 2 * n ** 2) + chs * 2 * n ** 2)
        jac = np.maximum(full - 1, 0)
        # algorithmic work: Q_c n^3 multiply-adds per Jacobian and per FP64 residual
        plain = np.sum(jac * 2 * wl.q_c * n ** 3)
        sysb = np.sum(full * (8 * n ** 2 + 4 * n * (n + 1)) + jac * 4 * n ** 2 + chs * (8 * n ** 2 + 4 * n))
        sliced = np.sum(np.maximum(it - 2, 0) * 2 * wl.q_c * n ** 3)
        # 1 ms per step: achieved = units / 1e-3 / scale
        assert np.isclose(rl["k_lu_mixed"]["achieved"], lu / 1e-3 / 1e12)
        assert np.isclose(rl["k_tc_gemm<plain>"]["achieved"], plain / 1e-3 / 1e12)
        assert np.isclose(rl["k_newton_system"]["achieved"], sysb / 1e-3 / 1e9)
        assert np.isclose(rl["k_tc_gemm<sliced>"]["achieved"], sliced / 1e-3 / 1e12)
        # the products issued: the FLOPs the kernels counted over the profiled time, reported
        # beside (never in) the algorithmic fraction
        assert np.isclose(rl["k_tc_gemm<plain>"]["issued_tflops"], 7.0e9 / 1e-3 / 1e12)
        assert np.isclose(rl["k_tc_gemm<sliced>"]["issued_tflops"], 3.0e10 / 1e-3 / 1e12)
        assert np.isclose(rl["k_tc_gemm<sliced>"]["issued_per_algorithmic"], 3.0e10 / sliced)
        assert np.isclose(rl["k_tc_gemm<sliced>"]["issued_frac"],
                          rl["k_tc_gemm<sliced>"]["issued_tflops"] / rl["k_tc_gemm<sliced>"]["peak"])
        assert "issued_tflops" not in rl["k_lu_mixed"]
        assert rl["k_tc_gemm<sliced>"]["work"] == "algorithmic"
        assert np.isclose(rl["k_tc_gemm<sliced>"]["frac"],
                          rl["k_tc_gemm<sliced>"]["achieved"] / rl["k_tc_gemm<sliced>"]["peak"])
    # the chord steps of the first two queries replace a factorisation by two triangular solves
    _, a, _ = bench.kernel_rooflines(1, wl, q, info, kprof, 1, np.full(4, True))
    _, b, _ = bench.kernel_rooflines(1, wl, q, info, kprof, 1, np.full(4, False))
    assert a["k_lu_mixed"]["achieved"] < b["k_lu_mixed"]["achieved"]


def test_chord_queries_follow_the_precision_and_switch(monkeypatch):
    wl = synth.WORKLOADS["sweep_n50"]
    q = synth.make_queries(wl, batch=5)
    assert bench.chord_queries(1, wl, q, []).all()
    assert not bench.chord_queries(0, wl, q, []).any()
    monkeypatch.setenv("RB_CHORD", "0")
    assert not bench.chord_queries(1, wl, q, []).any()


def test_combined_modes_are_exact_for_a_linear_pressure():
    """If the snapshots' pressures depend linearly on their velocities, p = M u, the combined
    basis built from them reconstructs M exactly (on the span of the snapshots: all of R^n)."""
    g = np.random.default_rng(4)
    n, m, K = 9, 5, 40
    U = g.standard_normal((K, n))
    M = g.standard_normal((m, n))
    P_hat, r = bench.combined_pressure_modes(U, U @ M.T)
    assert r == n
    np.testing.assert_allclose(P_hat, M, atol=1e-10)
    # rank-deficient snapshots: modes below the tolerance are dropped, the span is still exact
    U2 = g.standard_normal((K, 3)) @ g.standard_normal((3, n))
    P2, r2 = bench.combined_pressure_modes(U2, U2 @ M.T)
    assert r2 == 3
    np.testing.assert_allclose(U2 @ P2.T, U2 @ M.T, atol=1e-9)


def test_stratified_indices_cover_the_box():
    """Parity samples: one query per occupied cell of the alpha x log Re grid, the one nearest the
    cell's centre, so the sample spreads over the whole parameter box."""
    wl = synth.WORKLOADS["dense_n300"]
    q = synth.make_queries(wl)
    idx = synth.stratified_indices(wl, q.mu, cells=(6, 10))
    assert len(idx) == 60 and len(np.unique(idx)) == 60
    a = q.mu[idx, 0]
    r = np.log10(q.mu[idx, 1])
    ca = np.floor(a / 35.0 * 6).astype(int)
    cr = np.floor((r - 2.0) * 10).astype(int)
    assert len(set(zip(ca, cr))) == 60
    # nearest to the centre of its own cell
    for i, c1, c2 in zip(idx, ca, cr):
        d = ((q.mu[:, 0] / 35.0 * 6 - c1 - 0.5) ** 2 + ((np.log10(q.mu[:, 1]) - 2) * 10 - c2 - 0.5) ** 2)
        inside = (np.floor(q.mu[:, 0] / 35.0 * 6) == c1) & (np.floor((np.log10(q.mu[:, 1]) - 2) * 10) == c2)
        assert d[i] == d[inside].min()
