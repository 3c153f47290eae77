"""GB300-native (sm_103a) SCA+ADAM for the 2D ionic Hubbard model (arXiv 2311.04435).

The hot path (assemble, blocked pivoted LU / Gauss-Jordan inversion, log-det, adjoint
diag(G), gradient reduction, fused Adam) runs in the CUDA library ``libsca_gb300.so``
behind the C ABI of ``include/sca.h``; this package is its thin Python binding.
"""
from .api import (AdamConfig, Context, Params, Server, SolveResult, kernel_launches,  # noqa: F401
                  sca_potential, solve, version, workspace_bytes)
