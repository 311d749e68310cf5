"""The C ABI's contract on the GPU: BF16 storage of the convection tensors (RB_BF16) gives the
oracle's solution, and rb_solve_device / rb_solve_device_sized return once the solve is
enqueued (the stream's work is still running when the call comes back)."""
import dataclasses
import time

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bf16_storage_matches_oracle(rb, prec):
    """C and Cs handed over as BF16 bit patterns (2 bytes per value): velocity and pressure are
    the oracle's on the same values, and identical to loading the same values as FP32."""
    P = rb.RB_PREC_FP64 if prec == "fp64" else rb.RB_PREC_MIXED
    tol = 1e-10 if prec == "fp64" else TOL_MIXED
    wl = dataclasses.replace(synth.WORKLOADS["sweep_n50"], c_dtype="bf16")
    ops = synth.make_operators(wl, n_max=40)
    q = synth.make_queries(wl, batch=150, n_max=40)
    mu = np.concatenate([q.mu, synth.corner_queries(wl)])
    bits = rb.bf16_bits(ops.C)
    assert bits.dtype == np.uint16 and bits.nbytes * 2 == ops.C.nbytes
    o = oracle.Oracle.from_set(ops)
    u_ref, p_ref, _ = o.solve(mu, threads=8)
    with rb.Context(P) as ctx:
        ctx.load_set(ops)  # a BF16 workload goes in as RB_BF16
        u, p, info = ctx.rb_solve(mu)
    with rb.Context(P) as ctx:
        ctx.rb_load_operators(ops.A, ops.C, ops.f, ops.B, ops.As, ops.Cs, ops.fs)  # as FP32
        u32, p32, _ = ctx.rb_solve(mu)
    assert np.all(info["status"] == 0)
    assert rel(u, u_ref).max() <= tol
    assert rel(p, p_ref).max() <= 10 * tol
    np.testing.assert_array_equal(u, u32)
    np.testing.assert_array_equal(p, p32)


def test_bf16_rejects_non_bf16_values(rb):
    with pytest.raises(ValueError):
        rb.bf16_bits(np.array([1.0, 1.0 + 2.0 ** -10], dtype=np.float32))


def _blocked_enqueue(rb, ctx, torch, call):
    """Put a bounded spin kernel (about 0.3 s) on the stream, then make `call`: returns the host
    time of the call and whether an event recorded right after it had completed."""
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(6e8))  # a timed spin: ends by itself
        t0 = time.perf_counter()
        call(stream.cuda_stream)
        dt = time.perf_counter() - t0
        ev = torch.cuda.Event()
        ev.record(stream)
        done = ev.query()
        pending = ctx.rb_solve_device_status(wait=False)
    torch.cuda.synchronize()
    return dt, done, pending


@pytest.mark.parametrize("sized", [False, True])
def test_solve_device_returns_before_the_work_completes(rb, sized):
    import torch
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=50)
    q = synth.make_queries(wl, batch=1000, n_max=50)
    sizes = np.array([50, 24, 37, 9] * 250, dtype=np.int32) if sized else None
    dev = torch.device("cuda")
    d_mu = torch.from_numpy(q.mu).to(dev)
    d_n = torch.from_numpy(sizes).to(dev) if sized else None
    d_u = torch.empty((1000, 50), dtype=torch.float64, device=dev)
    d_p = torch.empty((1000, wl.m), dtype=torch.float64, device=dev)
    d_info = torch.empty((1000, 4), dtype=torch.float64, device=dev)
    with rb.Context(rb.RB_PREC_MIXED) as ctx:
        ctx.load_set(ops)
        u_ref, p_ref, info_ref = ctx.rb_solve(q.mu, n=sizes)

        def call(st):
            if sized:
                ctx.rb_solve_device_sized(d_mu, 1000, d_n, sizes, d_u, d_p, d_info, st)
            else:
                ctx.rb_solve_device(d_mu, 1000, d_n, d_u, d_p, d_info, st)

        # the first call of this batch shape tunes and captures the graph (synchronous)
        call(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert ctx.rb_solve_device_status(wait=True) == rb.RB_OK
        d_u.fill_(float("nan"))
        dt, done, pending = _blocked_enqueue(rb, ctx, torch, call)
        assert not done, "the call waited for the stream"
        assert pending == rb.RB_PENDING
        assert dt < 0.1, dt
        assert ctx.rb_solve_device_status(wait=True) == rb.RB_OK
    u = d_u.cpu().numpy()
    p = d_p.cpu().numpy()
    info = d_info.cpu().numpy().view(rb.INFO_DTYPE).reshape(1000)
    # the same solve as rb_solve's, up to the order of the sliced GEMM's FP64 atomic additions
    np.testing.assert_array_equal(info["status"], info_ref["status"])
    assert rel(u, u_ref).max() <= 1e-13
    assert rel(p, p_ref).max() <= 1e-12
