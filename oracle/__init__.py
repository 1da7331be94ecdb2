"""FP64 CPU oracle of PLAM / PCAL (Gao, Liu, Yuan, arXiv:1810.03930).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA path is checked against.  Only the test-suite, the
smoke check of the build entry point and the CPU-baseline leg of the benchmark
may import it; the library itself never calls it, and it shares no code with
the CUDA kernels (the two meet only in the seeded input generators of
`workloads`, which hold none of the method's arithmetic).

Layout
  objectives.py  f and grad f of the test problems (Section 5.2), FP64
  plam.py        the iteration of Algorithms 2 and 3 step by step, the
                 step-size rules of Section 5.1, the stopping test and the
                 final orthonormalisation (Section 5.3, Table "orth step")
  kernels.py     per-step reference values (Grams, multipliers, update,
                 column dots) for element-wise parity tests of single kernels
  moptqr.py      MOptQR, the comparison solver of Sections 5.3-5.4 (Table
                 "cost": projected gradient, Cholesky retraction, ABB step)

Parity status: every function here is pinned by a `-m "not gpu"` test against
closed forms, brute-force eigensolves, finite differences or invariants the
paper states, except the step-size sequence of the Barzilai-Borwein rules,
whose iterates the paper never prints: "parity unpinned" for `eta` values
beyond the invariants checked in tests/test_oracle_pins.py.
"""
from . import objectives, plam, kernels, moptqr  # noqa: F401
