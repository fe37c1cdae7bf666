"""CPU oracle for recursive fast matrix multiplication with diagonal scaling.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 restatement
of what Ballard, Benson, Druinsky, Lipshitz and Schwartz, "Improving the
numerical stability of fast matrix multiplication" (SIAM J. Matrix Anal.
Appl., 2016) defines.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it.  It shares no
code with the CUDA path in ``paper_1507_00687_gb300`` and imports nothing
from it.

Modules
-------
rules      coefficient matrices [[U, V, W]] as printed (App. A, App. B), the
           classical rules, the Winograd variant (derived, see its docstring),
           Brent equations, principal quantities (Sec. 4.1), rule transforms.
fmm        classical product, recursive stationary / uniform non-stationary
           fast multiplication (Eq. 3.2), Theorem 4.1 / 4.2 bounds, the
           componentwise quantity bounding the error in the proof of Thm 4.1.
scaling    outside (Alg. 1), inside (Alg. 2), repeated outside-inside
           (Alg. 3) scaling, real-valued and rounded to powers of two.
variants   the Castrapel-Gustafson variants of a <2,2,2> rule (Sec. 3.4) and
           random / round-robin / matrix-dependent selection per tree node.
precision  round-to-nearest-even emulation of bf16 / fp16 / e4m3 and the
           bf16 hi+lo split, written from the IEEE-754 definitions.
"""
