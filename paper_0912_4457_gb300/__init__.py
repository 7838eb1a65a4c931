"""Nested Krylov-Ritz evaluation of sgn(gamma5 D_w(mu)) b on one GB300.

The method is Bloch & Heybrock (2009), "A nested Krylov subspace method to
compute the sign function of large complex matrices".  The compute path is
the CUDA library ``libnksign.so`` (sources in ``csrc/``, C ABI in
``include/nksign.h``); ``nksign`` is its thin ctypes binding.
"""
from .nksign import (  # noqa: F401
    NK_ASYNC, NK_DOUBLE_PASS, NK_SHARED_P, NK_FP64, NK_MIXED, NK_NO_GRAPH, NK_PROFILE, NK_MAX_RHS, Context, Mlp, NkError,
    load_library,
)
