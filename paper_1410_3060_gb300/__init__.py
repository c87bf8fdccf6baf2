"""GB300-native temporally blocked 3D star-stencil sweeps (arXiv 1410.3060).

The compute path is the C-ABI library ``libstencil.so`` (hand-written
sm_103a CUDA kernels, declared in ``include/stencil.h``).  Python modules:

* ``stencil``    -- thin ctypes binding with the C names (``plan``,
  ``forward``, ``adjoint``, ...) taking torch device tensors;
* ``autograd``   -- ``WaveVarFn``: receiver-misfit loss with checkpointed
  forward and hand-written adjoint;
* ``workloads``  -- seeded synthetic inputs (no stencil arithmetic);
* ``perfmodel``  -- bytes/flops per lattice update and the paper's
  code-balance and cache-block models;
* ``build``      -- nvcc build of the library.

Importing the package loads nothing; ``stencil`` loads the library on first
use and raises if it is missing (there is no CPU fallback).
"""
