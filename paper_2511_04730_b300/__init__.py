"""B300-native LLOID hot path (SGNL, arXiv:2511.04730, Section II.C-D).

The compute path is the CUDA library ``liblloid_b300.so`` (C ABI in
``include/lloid.h``); this package holds its ctypes binding (``lloid``), the
offline SVD bank builder (``svdbank``) and the build script (``build``).
"""
from .lloid import Context, LloidError, TRIGGER_DTYPE, EVENT_DTYPE, Whitener, autotune  # noqa: F401
from .svdbank import SliceArrays, build_svd_bank  # noqa: F401
