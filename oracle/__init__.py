"""CPU FP64 oracle for the PDMCF method (Zhang & Boyd, "Solving Large Multicommodity
Network Flow Problems on GPUs").

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct reference that the
CUDA path is checked against. Only the test suite, the smoke check of the build entry
point and the CPU-baseline / reference legs of the benchmark may import it. The product
library never imports, links or calls anything here, and nothing here imports the
product library. The two share only the seeded input generators, which hold none of the
method's arithmetic.

Contents:
  pdmcf.py          Algorithm 2.1 step by step in float64 (dense F, Y; sparse A),
                    the sort-based capped-simplex projection of Sec. 2.6, the two
                    closed-form/root-equation proxes of Sec. 2.3, the residual of
                    Eq. (e-res), the primal weight rule of Eq. (e-primal_weight) and
                    the step size bound of Eq. (e-eta); plus the duality-gap and
                    relative KKT measures derived from the reduced Lagrangian (Eq. e-L).
  barrier.py        an independent log-barrier Newton solver for the compact problem
                    (Eq. e-compact-prob) on tiny instances, used only to pin pdmcf.py.
"""
