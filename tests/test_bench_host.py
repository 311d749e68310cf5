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
        _, rl, _ = bench.kernel_rooflines(1, wl, q, info, kprof, 1, np.full(4, chord))
        it = np.array([4, 4, 3, 2], float)
        full = np.minimum(it, 3) if chord else it
        chs = it - full
        lu = np.sum(full * (2 * n ** 3 / 3 + 2 * n ** 2) + chs * 2 * n ** 2)
        jac = np.maximum(full - 1, 0)
        plain = np.sum(jac * 6 * wl.q_c * n ** 3)
        sysb = np.sum(full * (8 * n ** 2 + 4 * n * (n + 1)) + jac * 4 * n ** 2 + chs * (8 * n ** 2 + 4 * n))
        sliced = np.sum(np.maximum(it - 2, 0) * 2 * n ** 2 * 21 * wl.q_c * n)
        # 1 ms per step: achieved = units / 1e-3 / scale
        assert np.isclose(rl["k_lu_mixed"]["achieved"], lu / 1e-3 / 1e12)
        assert np.isclose(rl["k_tc_gemm<plain>"]["achieved"], plain / 1e-3 / 1e12)
        assert np.isclose(rl["k_newton_system"]["achieved"], sysb / 1e-3 / 1e9)
        assert np.isclose(rl["k_tc_gemm<sliced>"]["achieved"], sliced / 1e-3 / 1e12)
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
