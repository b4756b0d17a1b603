"""CPU oracle for the cascading double-double GEMM.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the CUDA product path never
does, and this package never imports the product path.

* ``dd``      - the definition: C = A B in double-double, a scalar
                TwoProd/TwoSum triple loop in plain C (dd_oracle.c).
* ``cascade`` - the paper's approximation, step by step in numpy FP64
                (scales, Appendix A split, eq. Gemm10 bins, bin assembly).
"""
