"""GB300-native matrix-free elastic Lippmann-Schwinger solver (Shekhar et al., arXiv 2301.12836).

The method (frequency-domain volume integral equation for microseismic
wavefields in anisotropic elastic media, solved matrix-free by FFT and
BiCGSTAB) runs in hand-written CUDA kernels for sm_103a behind the C ABI of
``include/lsm.h``.  ``lsm`` is its Python binding; ``build`` compiles it.
"""
from . import lsm  # noqa: F401
from .lsm import (  # noqa: F401
    lsm_adjoint,
    lsm_apply,
    lsm_apply_c64,
    lsm_create,
    lsm_create_shared,
    lsm_default_opts,
    lsm_last_error,
    lsm_launch_count,
    lsm_solve,
    lsm_solve_batched,
    lsm_source,
)
