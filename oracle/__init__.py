"""CPU oracle for H-BACA (Liu, Sid-Lakhdar, Rebrova, Ghysels, Li: "A Parallel
Hierarchical Blocked Adaptive Cross Approximation Algorithm", arXiv 1901.06101).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 / complex128
restatement of the paper's algorithms, written to be checked against the paper
by eye.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The CUDA library never calls it, and it
shares no code with the CUDA library.

Modules
-------
sampler     counter-based SplitMix64 draws and the random initial column block
            (Alg. 1 line 1, Alg. 2 line 1).
generators  O(1) entry functions A(I, J) (Sec. 5 kernels; synthetic workloads).
linalg      greedy column-pivoted QR with explicit residual norms (Eq. QRIk,
            QRJk, LRID1), eps-rank of a truncated SVD (Sec. 2).
baca        ACA (Alg. 1), BACA (Alg. 2) with LRID / LRnorm / LRnormUp, and the
            SVD re-compression (Sec. 3.2, last paragraph).
hbaca       index trees and the hierarchical merge (Alg. 3, Eqs. columncomb,
            columnsvdmerge).

Parity status: every function here is pinned by tests under ``tests/`` marked
``not gpu`` (closed forms, brute force on tiny inputs, LAPACK special cases).
The BACA stopping rule itself is a heuristic (Eq. aca_stop): the bound
||A-UV||_F <= eps ||A||_F is an observation, not a theorem, so it is checked
with the slack stated in the tests.
"""
