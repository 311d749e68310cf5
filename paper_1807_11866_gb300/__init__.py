"""GB300-native online stage of the velocity-only reduced-basis method for steady
Navier-Stokes flow: C-ABI CUDA library (librb.so, include/rb.h) and its thin Python binding.

    from paper_1807_11866_gb300 import rb
    ctx = rb.Context(precision=rb.RB_PREC_MIXED)
    ctx.rb_load_operators(A, C, f, B, As, Cs, fs)
    u, p, info = ctx.rb_solve(mu)
"""
from . import rb  # noqa: F401
from ._build import build  # noqa: F401
