"""Oracle package: plain, slow CPU implementations of what the GPU path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs may import anything under ``oracle/``.  It shares no code
with the CUDA path.

  direct       FP64 direct sums of Eq. (rime) and its adjoint (C, threads).
  kernel_math  FP64 modified-ES kernel (Eq. semicircle2), its Fourier transform psi and
               the map error function l(x) of Eq. (maperror), used to reproduce the
               kernel-parameter table of App. A.
"""
