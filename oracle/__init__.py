"""FP64 CPU oracle for the separable low-rank Hankel (SHLR family) reconstruction.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, literal NumPy
(complex128) restatement of the paper's operators and ADMM algorithms
(Eqs. 2, 4-8, 13-17, S1-S9; Algorithms S1 and S2).  It shares no code,
tables or helpers with the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU baseline and
``--impl reference`` arm) may import it; the product path never does.

Modules
-------
transforms : centred unitary 1D DFT, the sparsifying-filter weights W and the
             Hankel multiplicity counts.
hankel     : Hankel lift H, its adjoint H*, the conjugate-flip (dagger) of
             Eq. 4, and the full row/column/PE/parameter lifts with their
             real adjoints.
svt        : singular value thresholding S_t via ``numpy.linalg.svd`` (Eqs. 16-17).
admm       : the X-update (Eq. 15 / S7) as a pointwise k-space divide, a dense
             normal-equation solve for tiny problems, and Algorithms S1 / S2.
metrics    : SSOS coil combination and RLNE (Eq. S10).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (see each test's docstring).
The paper's in-vivo RLNE/MSSIM figures cannot be reproduced without its data:
that comparison is "parity unpinned".
"""
from . import transforms, hankel, svt, admm, metrics  # noqa: F401
