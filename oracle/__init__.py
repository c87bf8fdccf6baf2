"""Plain FP64 CPU oracle for the stencil sweeps (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1410_3060_gb300``; the two meet only through the seeded
input generators in ``paper_1410_3060_gb300.workloads``.
"""
from .oracle import (  # noqa: F401
    J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA,
    RADIUS, NUM_ARRAYS, NUM_WEIGHTS, SECOND_ORDER,
    build, forward, forward_f32, adjoint, receiver_loss, loss_and_gradient, lib_path,
)
