"""Plain, slow, FP64 CPU oracle for SsNAL-EN (test infrastructure only).

This package is the correctness reference for the CUDA path.  It is written
from the paper (Boschi, Reimherr, Chiaromonte, "An Efficient Semi-smooth
Newton Augmented Lagrangian Method for Elastic Net", arXiv 2006.03970:
Secs. 2-3, Algorithm 1, Props. 1-2) and shares no code with
the CUDA path.  Only the test-suite, the smoke check of ``__graft_entry__``
and the CPU-baseline leg of ``bench.py`` may import it; the product path
never does.

Modules
-------
ssnal_en_ref : the SsNAL-EN algorithm step by step (Algorithm 1) plus the
               warm-started regularization path (Sec. 3.3).
checkers     : independent solution checkers used to pin the oracle:
               brute-force support enumeration, cyclic coordinate descent,
               closed forms, Elastic Net KKT conditions and the duality gap.
blas         : the thread count of the BLAS libraries the oracle runs on (one
               thread in the test-suite, so that no result depends on how a
               threaded BLAS splits its work).

Parity status
-------------
Every function that produces the final solution is pinned by the checkers
(tests/test_oracle_*.py).  The iterate path itself (iteration counts, the
active-set sizes per Newton step) is "parity unpinned": the paper prints no
iterates and no worked example.
"""
