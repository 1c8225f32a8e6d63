"""Plain FP64 CPU oracle for the NFFT-like procedure for bandlimited functions.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
reference that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path (``paper_2502_07155_gb300``)
never imports, calls or links it, and the two share no code: the only common
module is ``workloads`` (seeded input generators without any of the method's
arithmetic).

What it computes, step by step in the paper's order and notation:

* Algorithm 4.2 (NFFT-like procedure): step 0a window transform psi_hat by
  adaptive quadrature, step 1 precorrection, step 2 a DIRECT separable
  oversampled inverse DFT (no FFT), step 3 direct regularized-Shannon short
  sums over the closed index set J_{L,m}(x) of Eq. 4.8.
* Its adjoint D_psihat F^H Psi^T (the transpose of Eq. 4.11).
* Algorithm 2.1 (classical NFFT) with the periodized window and its adjoint.
* The NDFT of Eq. 2.1 by brute force.
* Node binning keys / stable permutation / tile offsets (an implementation
  device, defined here so that the GPU's integer results can be compared
  bit for bit).
* The derivative of the forward map with respect to the nodes.
* The tabulated (learned) window and its MLP parameterisation.

Pins (closed forms, invariants, brute force) live in ``tests/``.  Functions
whose values no pin fixes say "parity unpinned" in their docstring.
"""
from .nfft_oracle import *  # noqa: F401,F403
from .nfft_oracle import __all__  # noqa: F401
