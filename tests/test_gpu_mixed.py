"""GPU parity of the mixed-precision path (tensor-core Jacobian + FP64-accurate sliced residual)
against the FP64 CPU oracle, through the C ABI.

Tolerances: the converged velocity within 1e-8 relative L2 of the oracle per query (the bound
stated for mixed paths); the residual evaluated at a given u within 1e-12 of the size of its
terms (sum_j |A(mu)[k][j] u_j| + |C_mu(u,u)|-terms + |f|), which is what the FP64 stopping
rule needs; the Jacobian's convection part within 2^-12 of its magnitude (split BF16).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


def term_scale(o, ops, n, th, u):
    A, f = o.assemble(n, th)
    tc = th[o.q_a:o.q_a + o.q_c]
    Cabs = np.abs(ops.C[:, :n, :n, :n].astype(np.float64))
    conv = np.einsum("q,qjlk,j,l->k", np.abs(tc), Cabs, np.abs(u), np.abs(u))
    return np.abs(A) @ np.abs(u) + conv + np.abs(f)


@pytest.mark.parametrize("pairs", ["0", "1", "2"])
@pytest.mark.parametrize("n,qc,c_dtype", [(8, 3, "f64"), (50, 6, "f64"), (37, 4, "f32"),
                                          (64, 8, "bf16"), (72, 3, "f64")])
def test_eval_residual_and_jacobian(rb, n, qc, c_dtype, pairs, monkeypatch):
    """Residual and Jacobian at given u, with the GEMMs on single CTAs and on CTA pairs
    (256-row tiles; 256-column Jacobian tiles with a ragged last tile for n = 8, 37 and 72;
    with pairs = 2 and n >= 32 the sliced GEMM on 256-column tiles contracted chunk by chunk)."""
    monkeypatch.setenv("RB_GEMM_PAIRS", pairs)
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n, q_a=3, q_c=qc, c_dtype=c_dtype)
    o = oracle.Oracle.from_set(ops)
    g = np.random.default_rng(n)
    nq = 150  # more than one 128-row tile, ragged tail
    mu = np.stack([g.uniform(0, 35, nq), 10 ** g.uniform(2, 3, nq)], 1)
    u = g.standard_normal((nq, n)) * 0.05
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        R, J = ctx.rb_eval(mu, n, u, rb.RB_PREC_MIXED)
    for b in list(range(0, nq, 7)) + [nq - 1]:
        th = o.theta(*mu[b])
        Rr = o.residual(n, th, u[b])
        Jr = o.jacobian(n, th, u[b])
        A, _ = o.assemble(n, th)
        sc = term_scale(o, ops, n, th, u[b])
        assert np.max(np.abs(R[b] - Rr) / sc) <= 1e-12, b
        Jc, Jcr = J[b] - A, Jr - A
        # A(mu) enters the FP32 Jacobian rounded to FP32; the convection part comes from split
        # BF16 operands (hi*hi + hi*lo + lo*hi, about 16 significant bits)
        assert np.abs(Jc - Jcr).max() <= 2 ** -12 * np.abs(Jcr).max() + 2e-7 * np.abs(A).max()


@pytest.mark.parametrize("small", ["0", "1"])
@pytest.mark.parametrize("n", [2, 20, 50])
def test_sweep_parity(rb, n, small, monkeypatch):
    """Velocity and pressure of a sweep against the oracle; for n <= 32 through both the
    tensor-core pipeline (RB_SMALL=0) and the single-launch small-system solve (1)."""
    monkeypatch.setenv("RB_SMALL", small)
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n)
    q = synth.make_queries(wl, batch=200, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, inf_ref = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0), np.unique(info["status"], return_counts=True)
    assert np.all(info["precision_used"] == rb.RB_PREC_MIXED)
    assert rel(u, u_ref).max() <= TOL_MIXED
    assert rel(p, p_ref).max() <= 10 * TOL_MIXED


@pytest.mark.parametrize("n,nq,pairs", [(50, 300, "1"), (30, 130, "1"), (80, 300, "2")])
def test_cta_pair_gemms_solve(rb, n, nq, pairs, monkeypatch):
    """Whole solves (velocity and pressure) with both GEMMs restricted to CTA pairs (and, for
    pairs = 2, the 256-column sliced tiles): the tuner records them, and the result is the
    oracle's; batches not a multiple of 256 rows."""
    monkeypatch.setenv("RB_GEMM_PAIRS", pairs)
    monkeypatch.setenv("RB_SMALL", "0")  # the tensor-core pipeline also for n <= 32
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n)
    q = synth.make_queries(wl, batch=nq, n_max=n)
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(q.mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED, autotune=1) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(q.mu)
        tune = ctx.rb_tuning()
    assert tune and all(t["jacobian_gemm_cta_pairs"] and t["sliced_gemm_cta_pairs"] for t in tune)
    if pairs == "2":  # with pairs = 1 the tuner may pick either pair variant
        assert all(t["sliced_gemm_wide"] for t in tune)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL_MIXED
    assert rel(p, p_ref).max() <= 10 * TOL_MIXED


@pytest.mark.parametrize("n", [33, 64, 90, 100, 128])
def test_cta_elimination(rb, n, monkeypatch):
    """The CTA-per-query elimination (one row per thread, ceil(n / 32) warps, one barrier per
    pivot step) forced where it applies: velocity and pressure match the oracle."""
    monkeypatch.setenv("RB_ELIMINATION", "4")
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n, q_a=4, q_c=4)
    q = synth.make_queries(wl, batch=150, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
        tune = ctx.rb_tuning()
    assert all(t["elimination"].startswith("CTA") for t in tune if t["n_bucket"] > 32)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL_MIXED
    assert rel(p, p_ref).max() <= 10 * TOL_MIXED


@pytest.mark.parametrize("n,elim", [(20, ""), (50, ""), (72, ""), (40, "4"), (90, "4"),
                                    (120, "4"), (100, "2"), (150, "3")])
def test_chord_steps(rb, n, elim, monkeypatch):
    """Jacobian reuse from the second FP64-residual iteration on, with the factors kept by the
    warp-per-query elimination, by the CTA-per-query one (elim = 4; chord solve with 2, 3 or 4
    row slots) or by the blocked one (elim = 2, 3: 32- and 16-column panels, the forward
    substitution panel by panel with each panel's interchanges): the converged velocity and
    pressure are the oracle's with and without it, and it costs at most one extra iteration.
    The chord steps' residual is also taken as an increment on the previous one (RB_INCREMENT=1,
    the default) or as the full product (0): the same iterations and accuracy."""
    if elim:
        monkeypatch.setenv("RB_ELIMINATION", elim)
    monkeypatch.setenv("RB_SMALL", "0")
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=n)
    q = synth.make_queries(wl, batch=300, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(mu, threads=8)
    res = {}
    for chord, incr in (("0", "1"), ("1", "0"), ("1", "1")):
        monkeypatch.setenv("RB_CHORD", chord)
        monkeypatch.setenv("RB_INCREMENT", incr)
        with rb.Context(rb.RB_PREC_MIXED) as ctx:
            ctx.load_set(ops)
            res[chord + incr] = ctx.rb_solve(mu)
    for u, p, info in res.values():
        assert np.all(info["status"] == 0)
        assert rel(u, u_ref).max() <= TOL_MIXED
        assert rel(p, p_ref).max() <= 10 * TOL_MIXED
    assert np.all(res["11"][2]["iters"] <= res["01"][2]["iters"] + 1)
    # the chord steps' residual as an increment on the previous one (C quadratic: exact up to
    # the digit levels it keeps) costs no iteration and keeps the velocity at the full product's
    # accuracy
    assert np.array_equal(res["11"][2]["iters"], res["10"][2]["iters"])
    assert rel(res["11"][0], u_ref).max() <= 10 * max(rel(res["10"][0], u_ref).max(), 1e-13)


def test_issued_tensor_work_is_counted(rb, monkeypatch):
    """rb_profile_issued counts the MMAs the GEMM launches executed. With single-CTA tiles
    (128 x 128, K blocks of 64) and without chord steps every Jacobian launch issues the 3 split
    products and every residual launch the 15 digit pairs of S = 5 slices, over every K block
    of every output tile (padding included): exactly launches x tiles x products x K blocks x
    2 x 128 x 128 x 64 FLOPs."""
    for k, v in (("RB_SMALL", "0"), ("RB_AUTOTUNE", "0"), ("RB_GEMM_PAIRS", "0"), ("RB_CHORD", "0")):
        monkeypatch.setenv(k, v)
    wl = synth.WORKLOADS["sweep_n50"]
    n, nq = 40, 300
    ops = synth.make_operators(wl, n_max=n)
    mu = synth.make_queries(wl, batch=nq, n_max=n).mu
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        ctx.rb_solve(mu)
        ctx.rb_profile(True)
        _, _, info = ctx.rb_solve(mu)
        prof = ctx.rb_profile_read()
        issued = ctx.rb_profile_issued()
        ctx.rb_profile(False)
    assert np.all(info["status"] == 0)

    def up(a, b):
        return (a + b - 1) // b * b

    tiles = (up(nq, 128) // 128) * (up(n * n, 128) // 128)
    kb0 = up(wl.q_c * n, 64) // 64
    per_step = 2 * 128 * 128 * 64
    assert prof["k_tc_gemm<plain>"][1] > 0 and prof["k_tc_gemm<sliced>"][1] > 0
    assert issued["k_tc_gemm<plain>"] == prof["k_tc_gemm<plain>"][1] * tiles * 3 * kb0 * per_step
    assert issued["k_tc_gemm<sliced>"] == prof["k_tc_gemm<sliced>"][1] * tiles * 15 * kb0 * per_step
    assert issued["k_tc_gemm<sliced,pressure>"] > 0


@pytest.mark.parametrize("s1", ["7", "8"])
def test_pressure_linear_term_in_gemm_or_cuda_cores(rb, s1, monkeypatch):
    """As(mu) u of the pressure right-hand side (Eq. sup-vvar): from the sliced pressure GEMM's
    second K segment, theta^a digits against As digits (Q_a = 16 > 2 S1 with S1 = 7 slices), or
    in double-float on the CUDA cores (S1 = 8: 16 <= 2 S1). Both recover the oracle's pressure
    to rounding."""
    monkeypatch.setenv("RB_SMALL", "0")
    monkeypatch.setenv("RB_DIGITS_LINEAR", s1)
    wl = synth.WORKLOADS["sweep_n50"]
    n = 40
    ops = synth.make_operators(wl, n_max=n, q_a=16)
    q = synth.make_queries(wl, batch=300, n_max=n)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(mu, threads=8)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= TOL_MIXED
    assert rel(p, p_ref).max() <= 1e-10


def test_manufactured_mixed(rb):
    ops = synth.make_operators(synth.WORKLOADS["single_n20"])
    oracle.manufacture(ops, (10.0, 200.0))
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(np.array([[10.0, 200.0]]))
    assert info["status"][0] == 0
    assert rel(u[0], ops.u_star) <= TOL_MIXED


def test_nested_sizes_and_theta_user(rb):
    wl = synth.WORKLOADS["uneven_n120"]
    ops = synth.make_operators(wl, n_max=40, q_a=4, q_c=4)
    o = oracle.Oracle.from_set(ops)
    mu = synth.make_queries(wl, batch=130).mu
    sizes = np.array([1, 5, 17, 20, 39, 40] * 22)[:130].astype(np.int32)
    theta = np.stack([o.theta(*m) for m in mu])
    u_ref, _, _ = o.solve(mu, n=sizes, threads=8)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(mu, n=sizes)
        u2, _, info2 = ctx.rb_solve_theta(theta, n=sizes)
    assert np.all(info["status"] == 0) and np.all(info2["status"] == 0)
    assert rel(u, u_ref).max() <= TOL_MIXED
    assert rel(u2, u_ref).max() <= TOL_MIXED
    for b, n in enumerate(sizes):
        assert np.all(u[b, n:] == 0.0)


def test_status_codes_mixed(rb, monkeypatch):
    monkeypatch.setenv("RB_SMALL", "0")  # the tensor-core pipeline's statuses
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=12)
    mu = np.array([[10.0, 200.0], [20.0, 300.0], [1.0, 900.0]])
    with rb.Context(rb.RB_PREC_MIXED, max_iter=1) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(mu, n=np.array([12, 0, 13], dtype=np.int32))
    assert info["status"][0] == rb.RB_Q_NOT_CONVERGED and info["iters"][0] == 1
    assert info["status"][1] == rb.RB_Q_REJECTED and info["status"][2] == rb.RB_Q_REJECTED
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.rb_load_operators(np.zeros_like(ops.A), np.zeros_like(ops.C), ops.f)
        _, _, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == rb.RB_Q_SINGULAR)


def test_full_sweep_batch_sampled(rb):
    """The n = 50 sweep at its full batch (4096 queries) in mixed precision: a stratified
    sample of queries plus the corners against the oracle, and all of them against the FP64
    GPU path."""
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(mu)
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        ctx.load_set(ops)
        u64, p64, info64 = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0) and np.all(info64["status"] == 0)
    assert rel(u, u64).max() <= TOL_MIXED
    idx = np.concatenate([np.argsort(mu[:-4, 1])[:: len(mu) // 60][:60],
                          np.arange(len(mu) - 4, len(mu))])
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(mu[idx], threads=16)
    assert rel(u[idx], u_ref).max() <= TOL_MIXED
    assert rel(p[idx], p_ref).max() <= 10 * TOL_MIXED


@pytest.mark.parametrize("pairs", ["0", "2"])
@pytest.mark.parametrize("n,q,nq", [(160, 3, 130), (300, 2, 130)])
def test_large_n_mixed(rb, n, q, nq, pairs, monkeypatch):
    """Large Jacobians: sliced-GEMM tiles whose 128 columns hold fewer than one output row
    (n > 128), the blocked elimination (n = 160, 300); oracle on a sample. Single CTAs, and
    CTA pairs with the 256-column sliced tiles."""
    monkeypatch.setenv("RB_GEMM_PAIRS", pairs)
    wl = synth.WORKLOADS["dense_n300"]
    ops = synth.make_operators(wl, n_max=n, q_a=q, q_c=q, q_f=2)
    qs = synth.make_queries(wl, batch=nq - 2, n_max=n)
    mu = np.concatenate([qs.mu, synth.corner_queries(wl)[:2]])
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0)
    idx = np.array([0, nq // 2, nq - 1])
    o = oracle.Oracle.from_set(ops)
    u_ref, _, _ = o.solve(mu[idx], threads=8)
    assert rel(u[idx], u_ref).max() <= TOL_MIXED


def test_graph_and_stream_paths_agree(rb, monkeypatch):
    """The captured whole-solve graph (device-side while loop over FP64-residual iterations)
    gives the results of the stream path that checks convergence on the host after every
    iteration (identical but for the order in which the sliced GEMM's tiles add into the FP64
    residual with atomics: a few units in the last place); the graph is rebuilt when the batch
    changes, and honours the iteration cap."""
    monkeypatch.setenv("RB_SMALL", "0")
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=30)
    q = synth.make_queries(wl, batch=300, n_max=30)
    res = {}
    for g in (0, 1):
        with rb.Context(rb.RB_PREC_MIXED, use_graph=g) as ctx:
            ctx.load_set(ops)
            a = ctx.rb_solve(q.mu)
            b = ctx.rb_solve(q.mu[:77])          # another batch: graph rebuilt
            c = ctx.rb_solve(q.mu)               # back to the first
        res[g] = (a, b, c)
    for x, y in zip(res[0], res[1]):
        assert rel(x[0], y[0]).max() <= 1e-13 and rel(x[1], y[1]).max() <= 1e-12
        assert np.array_equal(x[2]["iters"], y[2]["iters"]) and np.array_equal(x[2]["status"], y[2]["status"])
    assert rel(res[1][0][0], res[1][2][0]).max() <= 1e-13
    assert rel(res[1][0][0][:77], res[1][1][0]).max() <= 1e-13
    with rb.Context(rb.RB_PREC_MIXED, use_graph=1, max_iter=3) as ctx:
        ctx.load_set(ops)
        _, _, info = ctx.rb_solve(q.mu[:50])
    assert np.all(info["iters"] <= 3)
    assert set(np.unique(info["status"])) <= {rb.RB_Q_OK, rb.RB_Q_NOT_CONVERGED}


def test_uneven_sizes_bucketed(rb):
    """Queries of sizes 20 / 40 / 80 / 120 (and 7, 97) from one n_max = 120 set of the uneven
    workload's shape (Q_a = Q_c = 8, C BF16-exact) run in size buckets inside one solve, in any
    order, and match the oracle."""
    wl = synth.WORKLOADS["uneven_n120"]
    ops = synth.make_operators(wl, n_max=120)  # the workload's Q_a = Q_c = 8, C BF16-exact
    q = synth.make_queries(wl, batch=48, n_max=120)
    rng = np.random.default_rng(5)
    sizes = rng.choice(np.array([20, 40, 80, 120, 7, 97], dtype=np.int32), size=48)
    o = oracle.Oracle.from_set(ops)
    u_ref, _, _ = o.solve(q.mu, n=sizes, threads=8)
    for g in (1, 0):
        with rb.Context(rb.RB_PREC_MIXED, use_graph=g) as ctx:
            ctx.load_set(ops)
            u, _, info = ctx.rb_solve(q.mu, n=sizes)
        assert np.all(info["status"] == 0)
        assert rel(u, u_ref).max() <= TOL_MIXED
        for b, n in enumerate(sizes):
            assert np.all(u[b, n:] == 0.0)


def test_autotuner_choices(rb):
    """The autotuner times the candidate variants of every bucket it meets and records a valid
    choice; with it off nothing is recorded. Either way the solution is the oracle's."""
    wl = synth.WORKLOADS["uneven_n120"]
    ops = synth.make_operators(wl, n_max=96, q_a=4, q_c=4)
    q = synth.make_queries(wl, batch=160, n_max=96)
    sizes = np.array([30, 96, 60, 12] * 40, dtype=np.int32)
    o = oracle.Oracle.from_set(ops)
    u_ref, _, _ = o.solve(q.mu, n=sizes, threads=8)
    with rb.Context(rb.RB_PREC_MIXED, autotune=1) as ctx:
        ctx.load_set(ops)
        u1, _, i1 = ctx.rb_solve(q.mu, n=sizes)
        tune = ctx.rb_tuning()
    with rb.Context(rb.RB_PREC_MIXED, autotune=0) as ctx:
        ctx.load_set(ops)
        u0, _, i0 = ctx.rb_solve(q.mu, n=sizes)
        assert ctx.rb_tuning() == []
    assert sorted(t["n_bucket"] for t in tune) == [16, 32, 64, 96]
    for t in tune:
        assert t["batch_class"] == 6  # 40 queries per bucket
        assert t["jacobian_gemm_stages"] in (4, 6, 7)
        assert t["sliced_gemm_stages"] in (4, 6, 7)
        if t["n_bucket"] > 80:
            assert t["elimination"].startswith("blocked") or t["elimination"].startswith("CTA")
        assert all(v > 0 for v in t["best_ms"].values())
    for u, info in ((u1, i1), (u0, i0)):
        assert np.all(info["status"] == 0)
        assert rel(u, u_ref).max() <= TOL_MIXED


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_maximum_sizes(rb, prec, monkeypatch):
    """The largest sizes the library accepts: n = RB_N_MAX (320) velocity modes, and m =
    RB_M_MAX (128) pressure modes (the CTA pressure solver), both against the oracle."""
    import dataclasses
    monkeypatch.setenv("RB_SMALL", "0")  # the mixed path's own pressure solver at m = 128
    P = rb.RB_PREC_FP64 if prec == "fp64" else rb.RB_PREC_MIXED
    tol = 1e-10 if prec == "fp64" else TOL_MIXED
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(dataclasses.replace(wl, q_b=0, m=0), n_max=320, q_a=1, q_c=1, q_f=1)
    q = synth.make_queries(wl, batch=3, n_max=320)
    o = oracle.Oracle.from_set(ops)
    u_ref, _, _ = o.solve(q.mu, threads=8)
    with rb.Context(P) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(q.mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= tol
    wlm = dataclasses.replace(wl, m=128, q_b=2)
    ops = synth.make_operators(wlm, n_max=20, q_a=2, q_c=2, q_f=2)
    q = synth.make_queries(wlm, batch=40, n_max=20)
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(q.mu, threads=8)
    with rb.Context(P) as ctx:
        ctx.load_set(ops)
        u, p, info = ctx.rb_solve(q.mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= tol
    assert rel(p, p_ref).max() <= 10 * tol


@pytest.mark.timeout(1200)
def test_dense_n300_full_batch_sampled(rb):
    """The n = 300 dense regime at its full size and in bench.py's configuration (16384 queries,
    Q = 24, C BF16-exact, one mixed-precision solve), with the last four queries replaced by the
    corners of the parameter box: every query converges, and 64 queries -- the four corners and
    60 stratified over alpha and log Re (the query nearest the centre of each cell of a 6 x 10
    grid) -- match the oracle."""
    wl = synth.WORKLOADS["dense_n300"]
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl)
    mu = q.mu.copy()
    mu[-4:] = synth.corner_queries(wl)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u, _, info = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0), np.unique(info["status"], return_counts=True)
    idx = np.concatenate([synth.stratified_indices(wl, mu[:-4]), np.arange(len(mu) - 4, len(mu))])
    assert len(idx) == 64
    o = oracle.Oracle.from_set(ops)
    u_ref, _, inf_ref = o.solve(mu[idx], threads=oracle.max_threads())
    assert np.all(inf_ref["status"] == 0)
    err = rel(u[idx], u_ref)
    assert err.max() <= TOL_MIXED, (idx[np.argmax(err)], err.max())
