"""FP64 CPU oracle for the CD-CCSD vvvv ladder (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the GPU
path computes.  It is used by the tests, by ``__graft_entry__.smoke`` and by
the CPU-baseline leg of ``bench.py``; the library itself never imports it.
It shares no code with the CUDA path.  See ``oracle.ladder`` for the
definitions and the passages of arXiv:2202.02019 they follow, and
``oracle.t1`` for the T1-transformed basis and the excited-state amplitudes.
"""
from .ladder import (  # noqa: F401
    tau, g_vvvv, residual_dense, residual_rows, residual_pm,
    gamma_dense, density_dense, density_rows, density_pm, dE_dL_general,
    dE_dtau, gamma_pm, lagrangian, euler_lagrangian, update_t2, sampled_rows,
)
