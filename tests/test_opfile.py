"""Operator files (the offline stage's output, Sec. 3.5-3.6): the writer's format read back by an
independent reader here, on the CPU; loading, and the refusal of damaged files, on the GPU."""
import os

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def rb():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb


def fnv1a_words(data: bytes) -> int:
    """FNV-1a 64 over 8-byte little-endian words, a last partial word zero-padded."""
    pad = (-len(data)) % 8
    words = np.frombuffer(data + b"\0" * pad, dtype="<u8")
    h = 0xCBF29CE484222325
    for w in words.tolist():
        h ^= w
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def read_file(path):
    raw = open(path, "rb").read()
    assert raw[:8] == b"RBOPS\0\0\0"
    version, hsize = np.frombuffer(raw[8:16], "<u4")
    n, m, q_a, q_c, q_f, q_b, dt = np.frombuffer(raw[16:44], "<i4")
    flags = int(np.frombuffer(raw[44:48], "<u4")[0])
    payload, csum = np.frombuffer(raw[48:64], "<u8")
    body = raw[64:]
    assert version == 1 and hsize == 64 and payload == len(body)
    assert csum == fnv1a_words(body)
    cdt = {0: np.float64, 1: np.float32, 2: np.uint16}[int(dt)]  # 2: BF16 bit patterns
    shapes = [((q_a, n, n), np.float64), ((q_c, n, n, n), cdt), ((q_f, n), np.float64)]
    if flags & 1:
        shapes += [((q_b, m, m), np.float64), ((q_a, m, n), np.float64), ((q_c, n, n, m), cdt),
                   ((q_f, m), np.float64)]
    out, off = [], 0
    for shp, t in shapes:
        cnt = int(np.prod(shp))
        out.append(np.frombuffer(body, t, cnt, off).reshape(shp))
        off += cnt * np.dtype(t).itemsize
    assert off == len(body)
    return out


def bf16_values(bits):
    """float32 values of BF16 bit patterns (independent of the binding's conversion)."""
    return (bits.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("c_dtype,pres", [("f64", True), ("f32", True), ("f64", False),
                                          ("bf16", True)])
def test_written_file_reads_back(rb, tmp_path, c_dtype, pres):
    import dataclasses
    wl = dataclasses.replace(synth.WORKLOADS["sweep_n50"], c_dtype=c_dtype)
    ops = synth.make_operators(wl, n_max=7, q_c=3)
    if not pres:
        ops.B = ops.As = ops.Cs = ops.fs = None
    path = tmp_path / "ops.rbops"
    rb.save_set(path, ops)
    arrs = read_file(path)
    want = [ops.A, ops.C, ops.f] + ([ops.B, ops.As, ops.Cs, ops.fs] if pres else [])
    assert len(arrs) == len(want)
    for a, w in zip(arrs, want):
        if a.dtype == np.uint16:  # BF16 storage: 2 bytes per value, the values unchanged
            a = bf16_values(a)
        np.testing.assert_array_equal(a, w)


def test_save_rejects_bad_sizes(rb, tmp_path):
    A = np.zeros((1, 3, 3))
    with pytest.raises(rb.RbError):
        rb.rb_save_operators(tmp_path / "x", A, np.zeros((0, 3, 3, 3)), np.zeros((1, 3)))
    with pytest.raises(rb.RbError):
        rb.rb_save_operators(tmp_path / "missing" / "x", A, np.zeros((1, 3, 3, 3)), np.zeros((1, 3)))


@pytest.mark.gpu
def test_loaded_file_solves_like_the_arrays(rb, tmp_path):
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=30)
    q = synth.make_queries(wl, batch=64, n_max=30)
    path = tmp_path / "ops.rbops"
    rb.save_set(path, ops)
    for prec in (rb.RB_PREC_FP64, rb.RB_PREC_MIXED):
        with rb.Context(prec) as ctx:
            ctx.load_set(ops)
            u1, p1, i1 = ctx.rb_solve(q.mu)
        with rb.Context(prec) as ctx:
            ctx.rb_load_operator_file(path)
            assert (ctx.n_max, ctx.m) == (30, wl.m)
            u2, p2, i2 = ctx.rb_solve(q.mu)
        assert np.all(i2["status"] == 0)
        np.testing.assert_allclose(u2, u1, rtol=0, atol=1e-13)
        np.testing.assert_allclose(p2, p1, rtol=0, atol=1e-12)


@pytest.mark.gpu
def test_damaged_files_are_refused(rb, tmp_path):
    wl = synth.WORKLOADS["sweep_n50"]
    ops = synth.make_operators(wl, n_max=9)
    good = tmp_path / "ops.rbops"
    rb.save_set(good, ops)
    raw = bytearray(open(good, "rb").read())
    cases = {}
    flipped = bytearray(raw)
    flipped[200] ^= 1
    cases["checksum"] = flipped
    cases["size"] = raw[:-8]
    wrong = bytearray(raw)
    wrong[8] = 7  # version
    cases["version"] = wrong
    with rb.Context(rb.RB_PREC_FP64) as ctx:
        for what, data in cases.items():
            path = tmp_path / f"{what}.rbops"
            open(path, "wb").write(bytes(data))
            with pytest.raises(rb.RbError) as e:
                ctx.rb_load_operator_file(path)
            assert what in str(e.value), (what, str(e.value))
        ctx.rb_load_operator_file(good)
        u, _, info = ctx.rb_solve(np.array([[10.0, 300.0]]))
        assert info["status"][0] == 0
