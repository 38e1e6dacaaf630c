"""Plain FP64 CPU oracle for the Léja-point log-determinant estimator (arXiv 2603.02207).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check in the repository's entry module
and the bench's CPU-baseline leg may import or run anything in this package; the library's
product path never does, and fails loudly when its CUDA extension is missing.

The oracle follows the paper's algorithms step by step, in the paper's order, with NumPy/SciPy
primitives (a sparse mat-vec, a Householder QR) as single steps and no blocking or fusion:

* leja.py      fast Léja points on [-2, 2]                       (Section 3, Eq. Léja5)
* divdiff.py   divided differences of log via Alg. 1              (Section 3.1, Algorithm 1)
* rng.py       counter-based SplitMix64 probe generator            (probe definition of this library)
* logdet.py    Gershgorin bounds, sigma-normalisation, Alg. 2 column by column, Hutch++
               (Algorithm 3), the frozen-basis gradient, and the scaled Newton-Léja reading.

It shares no code with the CUDA path. Every function has at least one pin in tests/ that does
not go through the function itself (closed forms, high-precision recurrences, brute force).
"""
